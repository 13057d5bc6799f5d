/*
 * labelfuse.h -- C ABI of the GB300 label-fusion library (liblabelfuse.so).
 *
 * Method: "Improving Semantic Image Segmentation via Label Fusion in
 * Semantically Textured Meshes" (arXiv 2111.11103).  For every camera frame
 * the triangle mesh is rendered with that frame's intrinsics and extrinsics
 * into a per-pixel row map (Sec. 3.3.1); every pixel's c-class probability
 * vector is added into the row of the texel it sees (Sec. 3.3.2,
 * Eq. texel-in-array) under one of the fusion rules (Eqs. sum, mul, maxsum
 * and their weighted forms, Sec. 3.2); the accumulators are normalised and
 * their arg max is the texel class (Sec. 3.2.1); finally the fused mesh is
 * rendered back into every view as a label image (Sec. 3.2.1, last paragraph).
 *
 * Conventions for every call:
 *   - Pointers named d_* are DEVICE pointers (cudaMalloc / PyTorch tensors on
 *     the current CUDA device), owned by the caller.  They are read-only
 *     unless the name ends in _out, and must stay valid until the work
 *     enqueued on `stream` has finished.  Pointers named h_* are host pointers.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  All device work is enqueued on it, asynchronously, unless the
 *     call's comment says it synchronises.  One sm_mesh must be used from one
 *     stream at a time (calls on one mesh are not thread-safe).
 *   - Arguments are validated before anything is enqueued; an invalid call
 *     returns SM_ERR_INVALID_ARG and changes nothing.  No call aborts the
 *     process or throws.  sm_last_error() gives a one-line reason for the
 *     calling thread's most recent failure.
 *   - Errors found by kernels (an out-of-range vertex index, a texel row past
 *     n_x) are latched in the mesh and returned by sm_check().
 *   - Layouts are C order (row-major).  Image coordinates: pixel (x, y) is
 *     sampled at image point (x, y), x to the right, y down; camera axes x
 *     right, y down, z forward.
 */
#ifndef LABELFUSE_H
#define LABELFUSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SM_API_VERSION 1
#define SM_MAX_CLASSES 254 /* label 255 is reserved for "no label" */
#define SM_MAX_IMAGE_DIM 16384
#define SM_MAX_TEXEL_RES 2048

typedef enum sm_status {
    SM_OK = 0,
    SM_ERR_INVALID_ARG = 1, /* bad size, null pointer, enum out of range */
    SM_ERR_OOM = 2,         /* a device allocation failed */
    SM_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    SM_ERR_STATE = 4,       /* call not allowed in the mesh's current state */
    SM_ERR_TIMEOUT = 5,     /* a bounded wait gave up */
    SM_ERR_INTERNAL = 6     /* a kernel latched an error (see sm_last_error) */
} sm_status;

/* Fusion rule, fixed per mesh at upload (the accumulators' meaning depends on it). */
typedef enum sm_rule {
    SM_RULE_SUM = 0,    /* f_sum, Eq. (sum) / (w-sum): A += w p                       */
    SM_RULE_LOGSUM = 1, /* f_mul, Eq. (mul) / (w-mul): A += w log(max(p, 2^-30))      */
    SM_RULE_MAXSUM = 2, /* f_maxsum, Eq. (maxsum) / (w-maxsum): A += w g(p), g keeps  */
                        /* the entries equal to max p and zeroes the others           */
    SM_RULE_VOTE = 3    /* one-hot vote: A += w onehot(first arg max p)               */
} sm_rule;

/* Pixel weights w_k (Sec. 3.2.2). */
typedef enum sm_weight {
    SM_WEIGHT_PIXEL = 0, /* w^(P) = 1: pixels are i.i.d. observations             */
    SM_WEIGHT_IMAGE = 1  /* w^(I) = 1 / |K_i ∩ K_x|: each image adds weight 1 to  */
                         /* every texel it sees                                    */
} sm_weight;

/* Storage type of the probability images. */
typedef enum sm_dtype {
    SM_F32 = 0,     /* float32, value = p                                  */
    SM_BF16 = 1,    /* bfloat16 q with a float32 scale per pixel, p = q*s  */
    SM_FP8_E4M3 = 2 /* fp8 e4m3 q with a float32 scale per pixel, p = q*s  */
} sm_dtype;

/* Pinhole intrinsics in pixels. */
typedef struct sm_intrinsics {
    double fx, fy, cx, cy;
} sm_intrinsics;

/* Opaque mesh + accumulator state, owned by the library. */
typedef struct sm_mesh sm_mesh;

/* ------------------------------------------------------------------------ */

/* Uploads a triangle mesh and allocates its accumulators (Sec. 3.1, 3.3.2).
 *
 *   d_vertices  V x 3 float32 world coordinates (metres), device.
 *   d_faces     F x 3 int32 vertex indices, device.  Indices outside [0, V)
 *               are latched as SM_ERR_INTERNAL (sm_check) and the face is
 *               never drawn.
 *   d_texel_res F int32 texel steps s_t >= 1 (|X_t| = (s^2+s)/2 texels,
 *               Sec. 3.1), device; NULL means s = 1 for every triangle
 *               (gamma = 0, one row per triangle).  For s > 1 the uv origin is
 *               the vertex with the interior angle closest to 90 degrees.
 *               s outside [1, SM_MAX_TEXEL_RES] -> SM_ERR_INVALID_ARG.
 *   n_classes   c in [1, SM_MAX_CLASSES].
 *   rule, weight  fusion rule and pixel weight used by every later fusion.
 *   *out        receives the mesh; free it with sm_mesh_free.
 *
 * The library copies the geometry, so the caller may free its buffers once
 * the call returns.  Rows are stacked triangle by triangle: the row of texel
 * x on triangle t is l = id_t + id_x (Eq. texel-in-array), id_t the prefix sum
 * of the texel counts.  n_x must stay below 2^31.  The accumulators start at
 * zero.  Synchronises `stream` (it reads n_x back).
 * Errors: SM_ERR_INVALID_ARG, SM_ERR_OOM, SM_ERR_CUDA. */
sm_status sm_mesh_upload(const float *d_vertices, int64_t V, const int32_t *d_faces, int64_t F,
                         const int32_t *d_texel_res, int32_t n_classes, sm_rule rule, sm_weight weight,
                         void *stream, sm_mesh **out);

/* Renders and fuses N frames into the mesh's accumulators (Sec. 3.3.1-3.3.2).
 *
 *   d_probs   N x H x W x c probabilities, pixel-major (the c values of a pixel
 *             are contiguous), device, in `dtype`.  16-byte aligned.
 *   d_scale   N x H x W float32 per-pixel scales for BF16/FP8, NULL for F32.
 *   d_K       N intrinsics, device.
 *   d_cam_to_world  N x 16 float64 row-major camera-to-world poses, device
 *             (rigid: the world-to-camera rotation is the transpose).
 *   N, H, W   frame count (0 is a no-op) and image size, 1..SM_MAX_IMAGE_DIM.
 *   d_idmap_out  N x H x W int32 row map of every frame (-1 = no triangle), or
 *             NULL.  Row maps are deterministic (see below).
 *
 * Renderer: vertices are projected in binary32 and snapped to 1/256 pixel; a
 * triangle with any vertex at depth <= 0.05 is dropped; coverage is decided
 * by exact integer edge functions with a top-left fill rule; the nearest
 * surface wins by 1/z interpolated in binary32, an exact tie going to the
 * lower triangle index.  Accumulation is float32 with atomics, so results
 * agree with an exact sum up to rounding.  The rows' observation counts are
 * kept alongside the accumulators.
 * Scratch: the mesh keeps a z-buffer (two slots of one launch's frames, 8
 * bytes per pixel) and, for image weights, per-frame row histograms, grown on
 * demand and in compressible device memory where the GPU offers compute data
 * compression (see sm_device_alloc).  Replacing a compressible buffer by a
 * larger one waits for the device to be idle (only when a call needs more
 * than every earlier call on the mesh); inside a stream capture the library
 * takes stream-ordered memory instead.
 * Errors: SM_ERR_INVALID_ARG, SM_ERR_OOM, SM_ERR_CUDA, SM_ERR_STATE (mesh
 * freed). */
sm_status sm_fuse_frames(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                         const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N, int32_t H, int32_t W,
                         int32_t *d_idmap_out, void *stream);

/* Normalises the accumulators and takes the arg max (Sec. 3.2.1).
 *
 *   d_dist    n_x x c float32 fused distributions (L1-normalised; for the
 *             log-sum rule exp(L - max L) / sum exp(L - max L)), or NULL.
 *   d_labels  n_x int32 arg max per row (lowest class on ties), -1 for rows
 *             never observed, or NULL.
 * Also stores the labels inside the mesh for sm_render_*.  Rows never
 * observed get an all-zero distribution.
 * Errors: SM_ERR_CUDA. */
sm_status sm_normalise(sm_mesh *m, float *d_dist, int32_t *d_labels, void *stream);

/* Renders the fused labels into N views given by their poses (the fused mesh
 * rendered from the original poses, Sec. 3.2.1).
 *
 *   d_labels_out  N x H x W uint8 class per pixel; 255 where no triangle is
 *                 seen or the row was never observed.
 *   d_idmap_out   N x H x W int32 row maps, or NULL.
 * Requires an earlier sm_normalise (else SM_ERR_STATE). */
sm_status sm_render_labels(sm_mesh *m, const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N,
                           int32_t H, int32_t W, uint8_t *d_labels_out, int32_t *d_idmap_out, void *stream);

/* Render-back from row maps kept from sm_fuse_frames (no second raster):
 * d_labels_out[k] = label of row d_idmap[k], 255 for -1 or unobserved rows.
 * Requires an earlier sm_normalise (else SM_ERR_STATE). */
sm_status sm_render_idmap(sm_mesh *m, const int32_t *d_idmap, int64_t n_pixels, uint8_t *d_labels_out,
                          void *stream);

/* End to end from host memory: fuses N frames whose predictions, scales and
 * cameras are in HOST memory (pinned memory lets the copies overlap the
 * work), then normalises and renders every frame's label image back into
 * host memory.  Equivalent to copying the inputs to the device and calling
 * sm_fuse_frames, sm_normalise and sm_render_idmap, but streamed: frames move
 * host -> device in batches on a copy stream, double-buffered, while the
 * previous batch is rendered and fused; row maps stay on the device.
 *
 *   h_probs        N x H x W x c in `dtype` (host), h_scale N x H x W (host,
 *                  BF16/FP8 only), h_K N intrinsics, h_cam_to_world N x 16.
 *   h_labels_out   N x H x W uint8 (host), 255 = no label.
 * Accumulates into the mesh's current state (call sm_reset first for a fresh
 * fusion).  Synchronises `stream` before returning.  Library-owned staging
 * (two batches of predictions, the row maps and label images of all N
 * frames) is allocated on first use and kept.
 * Errors: SM_ERR_INVALID_ARG, SM_ERR_OOM, SM_ERR_CUDA. */
sm_status sm_fuse_render_host(sm_mesh *m, const void *h_probs, sm_dtype dtype, const float *h_scale,
                              const sm_intrinsics *h_K, const double *h_cam_to_world, int32_t N, int32_t H, int32_t W,
                              uint8_t *h_labels_out, void *stream);

/* Image-weight mix (Fig. 5a): for a mesh uploaded with SM_WEIGHT_IMAGE, every
 * later fusion weighs a pixel whose row holds n pixels of its frame by
 * (1 - alpha) + alpha / n, evaluated in binary32.  alpha = 1 (the default) is
 * w^(I) of Sec. 3.2.2, alpha = 0 gives weight 1 as w^(P); the paper plots the
 * interpolation without printing its form, and this linear mix is the
 * project's reading.  Host-side setting, nothing is enqueued.
 * Errors: SM_ERR_INVALID_ARG (NULL mesh, a w^(P) mesh, alpha outside [0, 1]). */
sm_status sm_set_weight_mix(sm_mesh *m, float alpha);

/* Texel steps from gamma (Sec. 3.1): s_t = max(1, ceil(gamma sqrt(a_t))), with
 * a_t read as the largest number of pixels on which triangle t is the visible
 * surface in any one of the N frames (the paper's "area in pixels" does not
 * say over which views).  A visibility pre-pass over the frames (the same
 * raster as sm_fuse_frames) gives a_t; the square root and product are
 * evaluated in binary32, correctly rounded.  m must have been uploaded
 * without texel steps (one row per triangle); the result feeds the
 * d_texel_res argument of a second sm_mesh_upload.
 *
 *   d_K, d_cam_to_world  N frames, as for sm_fuse_frames (device).
 *   gamma                in [0, 64]; 0 gives s_t = 1 everywhere.
 *   d_area_out           F int32 a_t, or NULL.
 *   d_texel_res_out      F int32 s_t (device, required).
 * Leaves the mesh's accumulators untouched.
 * Errors: SM_ERR_INVALID_ARG, SM_ERR_STATE (a texel-mode mesh), SM_ERR_OOM,
 * SM_ERR_CUDA. */
sm_status sm_texel_res_from_gamma(sm_mesh *m, const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N,
                                  int32_t H, int32_t W, float gamma, int32_t *d_area_out, int32_t *d_texel_res_out,
                                  void *stream);

/* Frames per launch of the two-stream path (the paper has no counterpart: a
 * throughput setting of this implementation; results do not depend on it):
 * later calls on this mesh with frames of H x W pixels raster and scatter
 * that many frames per launch pair, as if sm_autotune_batch had chosen it.
 * frames = 0 restores the default (about 48 MB of z-buffer per launch).
 *   frames   0, or a multiple of 4 in [4, 1024].
 * Errors: SM_ERR_INVALID_ARG. */
sm_status sm_set_launch_frames(sm_mesh *m, int32_t H, int32_t W, int32_t frames);

/* Frames of one scene for sm_fuse_scenes: the arguments of sm_fuse_frames
 * (device pointers, same layouts) for one mesh. */
typedef struct sm_scene_frames {
    sm_mesh *mesh;
    const void *d_probs;            /* N x H x W x c, HWC, dtype; 16-byte aligned */
    sm_dtype dtype;
    const float *d_scale;           /* N x H x W, NULL iff SM_F32 */
    const sm_intrinsics *d_K;       /* N */
    const double *d_cam_to_world;   /* N x 16 row-major */
    int32_t N, H, W;
    int32_t *d_idmap_out;           /* N x H x W or NULL */
} sm_scene_frames;

/* Fuses the frames of many independent scenes, each into its own mesh, as
 * sm_fuse_frames would one after another (Sec. 3.3.1 and 3.3.2 per scene;
 * batching many scenes is a throughput setting of this implementation, the
 * paper has no counterpart).  Scenes whose meshes have no texel steps, pixel
 * weights w^(P) and c = 20 or 40 go through the persistent work-queue kernel:
 * those with the same class count, storage type and rule share one launch
 * (up to 12 scenes; plus one launch for the frames past their last full
 * batch), whose CTAs take (scene, frame batch) raster and scatter items from
 * a device queue, so uneven scenes leave no launch tails between them.  The
 * queue shape of each scene is its mesh's (sm_set_queue_shape or
 * sm_autotune_batch for its frame size, else the defaults).  Other scenes are
 * fused by sm_fuse_frames on the same stream.  Meshes must be distinct and on
 * one device.  Everything is enqueued on `stream`; results per scene equal
 * sm_fuse_frames'.
 * Errors: SM_ERR_INVALID_ARG (NULL, shared mesh, meshes on different devices,
 * n > 1024, any argument sm_fuse_frames would refuse, reported with the
 * scene's index), SM_ERR_OOM, SM_ERR_CUDA. */
sm_status sm_fuse_scenes(const sm_scene_frames *scenes, int32_t n, void *stream);

/* Launch path and shape of the fusion (the paper has no counterpart: a
 * throughput setting of this implementation; results do not depend on it).
 * By default sm_fuse_frames takes the two-stream path: per batch of frames a
 * raster launch (cluster cull + raster) on a second stream and a persistent
 * scatter launch.  For a mesh uploaded without texel steps, with pixel
 * weights w^(P) and c = 20 or 40, a non-zero frames_per_batch switches the
 * mesh to the work-queue path: one persistent kernel per call takes work
 * items from a device queue, raster items (one frame, raster_rounds x 1,152
 * clusters of 32 faces) running `lookahead` batches ahead of scatter items
 * (scatter_tiles tiles of 256 pixels) and spread evenly among them, so that
 * raster and scatter share the SMs without a launch boundary between batches.
 * The shape applies to later calls with frames of H x W pixels (other sizes
 * take the defaults).  frames_per_batch = 0 returns the mesh to the
 * two-stream path.
 *   frames_per_batch  0, or a multiple of 4 in [4, 128]  (default 32)
 *   lookahead         [1, 4]                               (default 2)
 *   raster_rounds     [1, 64]                              (default 1)
 *   scatter_tiles     [1, 4096]                            (default 128)
 * Errors: SM_ERR_INVALID_ARG. */
sm_status sm_set_queue_shape(sm_mesh *m, int32_t H, int32_t W, int32_t frames_per_batch, int32_t lookahead,
                             int32_t raster_rounds, int32_t scatter_tiles);

/* Autotuner of the launch path and shape (the paper has no counterpart: a
 * throughput setting of this implementation).  Tunes the frames per launch
 * of the two-stream path: fuses the given frames twice per candidate batch
 * size (4 to 1,024 frames spaced by about a quarter, whole launches of at
 * most N frames, both z-buffer slots within 8 GB; the first pass sizes the
 * scratch buffers) and times the second on `stream`
 * with CUDA events.  For a mesh that the work-queue path applies to (see
 * sm_set_queue_shape) it then tunes the queue's shape one parameter at a
 * time from its defaults (frames per batch in {8, 16, 24, 32, 48, 64},
 * lookahead in {1, 2, 3}, raster rounds in {1, 2, 4}, scatter tiles in {32,
 * 64, 128, 256}) and keeps whichever path has the faster per-frame time.
 * Later calls on this mesh with frames of H x W pixels use the choice
 * (results do not depend on it).  Synchronises `stream`; resets the
 * accumulators (P and counts are zero afterwards).  *best_out, if not NULL,
 * receives the chosen frames per launch (or per batch of the queue).
 *   d_probs ...  N >= 4 frames as for sm_fuse_frames (a representative
 *                sample; a launch size is timed only on whole launches,
 *                so sizes near N are timed without the overlap of
 *                consecutive launches).
 * Errors: SM_ERR_INVALID_ARG, SM_ERR_OOM, SM_ERR_CUDA. */
sm_status sm_autotune_batch(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                            const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N, int32_t H, int32_t W,
                            int32_t *best_out, void *stream);

/* Fusion with explicit per-pixel weights: as sm_fuse_frames, but pixel k of
 * the N frames weighs d_weights[k] (N x H x W float32, device) in the
 * weighted rules (Sec. 3.2.2, Eqs. w-sum / w-mul / w-maxsum), replacing the
 * mesh's own weight (w^(P) or w^(I)).  Used with the learned confidence below.
 * Errors: as sm_fuse_frames, SM_ERR_INVALID_ARG for NULL weights. */
sm_status sm_fuse_frames_weighted(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                                  const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N, int32_t H,
                                  int32_t W, const float *d_weights, int32_t *d_idmap_out, void *stream);

/* Learned per-observation confidence: the weight of an observation predicted
 * by a small network (an extension of the weights of Sec. 3.2.2; the paper's
 * weights are fixed).
 *
 * Features (SM_CONF_FEATURES per pixel, float32): |cos| between the visible
 * triangle's normal and the pixel's viewing ray; depth of the visible surface
 * (1 / interpolated 1/z) / 4 m; prediction entropy -sum p ln max(p, 2^-30) /
 * ln c; top-2 margin p(1) - p(2); distance to the nearest image border /
 * (min(H, W) / 2).  Background pixels get zeros.
 * Network: 5 -> 32 -> 32 -> 1, ReLU, linear output o: the log-odds that the
 * observation agrees with the fused label.  Fusion weight w = max(o, 1/16),
 * the log-odds weight of an independent two-way vote (Nitzan and Paroush,
 * 1982) clipped at a small floor (a row whose every observation is predicted
 * below even odds keeps the plain vote).  SM_CONF_PARAMS float32
 * parameters in the order W1 (32 x 5, row = output), b1, W2 (32 x 32), b2,
 * w3 (32), b3, used rounded to bfloat16 with float32 accumulation.
 * Training: mean binary cross-entropy of sigmoid(o) against targets
 * y in {0, 1}. */
#define SM_CONF_FEATURES 5
#define SM_CONF_PARAMS 1281

/* Renders the N frames and writes every pixel's features (d_feat_out,
 * N x H x W x SM_CONF_FEATURES float32) and row (d_rows_out, N x H x W int32,
 * -1 for background).  Inputs as for sm_fuse_frames; both outputs are
 * caller-owned device buffers.  Leaves the accumulators untouched.
 * Errors: SM_ERR_INVALID_ARG (NULL mesh or pointer, sizes, a scale given for
 * F32 or missing for BF16/FP8), SM_ERR_OOM, SM_ERR_CUDA. */
sm_status sm_conf_features(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                           const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N, int32_t H, int32_t W,
                           float *d_feat_out, int32_t *d_rows_out, void *stream);

/* Learned confidence inference in one pass (an extension of the weighted
 * rules of Sec. 3.2.2; the paper has no counterpart): renders the N frames
 * (as sm_fuse_frames) and, per pixel, computes the five features of
 * sm_conf_features and the network's weight w = max(o, 1/16) of
 * sm_conf_forward, without writing the features out.  The 32 x 32 hidden
 * layer runs on the tensor cores with its inputs (the first layer's ReLU
 * activations) rounded to bfloat16 and float32 accumulation, so w differs
 * from sm_conf_forward's by that rounding (about 4e-3 at most).
 *   d_params     SM_CONF_PARAMS float32 (device).
 *   d_w_out      N x H x W float32: w, 0 for background pixels.
 *   d_rows_out   N x H x W int32: the row map (-1 = background).
 * The result feeds sm_fuse_frames_weighted.  Leaves the accumulators
 * untouched.  Errors: SM_ERR_INVALID_ARG, SM_ERR_OOM, SM_ERR_CUDA. */
sm_status sm_conf_weights(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                          const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N, int32_t H, int32_t W,
                          const float *d_params, float *d_w_out, int32_t *d_rows_out, void *stream);

/* Confidence-weighted fusion with one raster pass per frame: per batch of
 * frames, the raster, then the weights of sm_conf_weights computed from the
 * batch's z-buffer (the same kernel, the same w bit for bit), then the
 * scatter of sm_fuse_frames_weighted with those weights.  The result equals
 * sm_conf_weights followed by sm_fuse_frames_weighted (up to the order of
 * the float32 additions), without the second raster pass and the full-size
 * weight buffer.  Inputs as for sm_fuse_frames, plus
 *   d_params     SM_CONF_PARAMS float32 (device).
 *   d_w_out      optional N x H x W float32: receives w (0 for background).
 *   d_idmap_out  optional N x H x W int32: receives the row map.
 * Keeps one batch of weights (frames per launch x H x W float32) in the
 * mesh's scratch.  Errors: as sm_fuse_frames_weighted, SM_ERR_INVALID_ARG
 * for a NULL d_params. */
sm_status sm_fuse_frames_confident(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                                   const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N, int32_t H,
                                   int32_t W, const float *d_params, float *d_w_out, int32_t *d_idmap_out,
                                   void *stream);

/* Training targets: d_target_out[k] = 1 where pixel k's first arg max equals
 * the fused label of its row d_rows[k], else 0 (background, unseen rows).
 * d_probs n_pixels x c in `dtype` (+ d_scale n_pixels float32 for BF16/FP8),
 * d_rows n_pixels int32, d_target_out n_pixels float32, all device.
 * Requires an earlier sm_normalise.
 * Errors: SM_ERR_INVALID_ARG (NULL mesh or pointer, n_pixels < 0, dtype),
 * SM_ERR_STATE (no sm_normalise since the last fusion), SM_ERR_CUDA. */
sm_status sm_conf_targets(sm_mesh *m, const void *d_probs, sm_dtype dtype, const float *d_scale,
                          const int32_t *d_rows, int64_t n_pixels, float *d_target_out, void *stream);

/* Inference: d_w_out[i] = max(MLP(d_feat[i]), 1/16) for n observations.
 * d_params SM_CONF_PARAMS float32, d_feat n x SM_CONF_FEATURES float32,
 * d_w_out n float32, all device; n == 0 is a no-op.
 * Errors: SM_ERR_INVALID_ARG (n < 0, NULL pointer), SM_ERR_CUDA. */
sm_status sm_conf_forward(const float *d_params, const float *d_feat, int64_t n, float *d_w_out, void *stream);

/* One gradient-descent step on the mean binary cross-entropy of n
 * observations: d_grad_out (SM_CONF_PARAMS, required) receives the gradient
 * with respect to the bfloat16-rounded parameters, d_loss_out (1 float,
 * required) the loss before the step, and d_params -= lr * gradient.
 * d_feat n x SM_CONF_FEATURES and d_target n float32; all device.
 * Reproducible: the sums over observations are exact 64-bit fixed-point sums
 * (resolution 2^-40) of per-block float32 partial sums, so the same inputs
 * give the same gradient, loss and parameters bit for bit on one GPU model.
 * A partial sum that is not finite, or of magnitude 2^22 or more, makes the
 * gradient and loss NaN.  Takes (SM_CONF_PARAMS + 2) x 8 bytes from the
 * device's stream-ordered memory pool for the duration of the call.
 * Errors: SM_ERR_INVALID_ARG (n < 0, lr NaN or outside [0, 1e6), NULL
 * pointer), SM_ERR_OOM (the pool allocation failed), SM_ERR_CUDA. */
sm_status sm_conf_train_step(float *d_params, const float *d_feat, const float *d_target, int64_t n, float lr,
                             float *d_grad_out, float *d_loss_out, void *stream);

/* The same step on a minibatch given by indices (a stochastic-gradient step
 * over the observations the agreement targets label; the paper has no
 * counterpart): the i-th observation of the minibatch (i < m) is observation
 * d_idx[i] of the n_obs rows of d_feat (n_obs x SM_CONF_FEATURES float32) and
 * d_target (n_obs float32), and the loss and gradient are means over the m.
 * d_idx: m int64 indices, device, drawn by the caller (repeats allowed).  The
 * rows are read where they lie, so the call gives bit for bit what
 * sm_conf_train_step gives on the gathered rows.  An index outside [0,
 * n_obs) is not read and makes the step's gradient and loss NaN, as a
 * non-finite partial sum does.
 * Errors: SM_ERR_INVALID_ARG (m < 0, n_obs < 0, m > 0 with n_obs = 0, lr NaN
 * or outside [0, 1e6), NULL pointer), SM_ERR_OOM, SM_ERR_CUDA. */
sm_status sm_conf_train_step_indexed(float *d_params, const float *d_feat, const float *d_target, int64_t n_obs,
                                     const int64_t *d_idx, int64_t m, float lr, float *d_grad_out, float *d_loss_out,
                                     void *stream);

/* Page-locked host memory for the host buffers of sm_fuse_render_host (the
 * paper has no counterpart: this is plumbing of the host path).  Memory from
 * here is copied to the device at the host link's full rate in one piece,
 * whatever its size; some runtimes pin very large tensors in ways that copy
 * markedly slower.  *out receives bytes > 0 bytes of host memory, owned by the
 * caller until sm_host_free(*out).
 * Errors: SM_ERR_INVALID_ARG (NULL out, bytes == 0), SM_ERR_OOM. */
sm_status sm_host_alloc(uint64_t bytes, void **out);
sm_status sm_host_free(void *p);

/* Device memory for the buffers the path writes and later reads in runs of
 * equal or similar values -- the row maps kept between sm_fuse_frames and
 * sm_render_idmap, and label images -- in compressible memory (the paper has
 * no counterpart: this is plumbing of the memory system).  With
 * SM_DEVICE_COMPRESSIBLE, and where the GPU and driver offer compute data
 * compression, the memory system keeps such data compressed in DRAM, so
 * writing and reading it moves fewer bytes; otherwise (or with flags 0) the
 * block is ordinary device memory.  The library holds its own z-buffer, row
 * histograms and internal row maps in the same memory; with the environment
 * variable LABELFUSE_COMPRESSIBLE_MEMORY=0 it uses ordinary memory
 * everywhere.  *out receives `bytes` > 0 bytes on `device`, uninitialised,
 * owned by the caller until sm_device_free(*out);
 * *compressed_out (may be NULL) is 1 if the block is compressible.  Any
 * kernel, copy or memset may use the block.  Both calls are synchronous;
 * sm_device_free first waits for the block's device to be idle (no work may
 * still use the block), so neither belongs inside a stream capture.
 * Errors: SM_ERR_INVALID_ARG (NULL out, bytes == 0, unknown flags, no such
 * device, a pointer that sm_device_alloc did not return), SM_ERR_OOM,
 * SM_ERR_CUDA. */
#define SM_DEVICE_COMPRESSIBLE 1
sm_status sm_device_alloc(int32_t device, uint64_t bytes, int32_t flags, void **out, int32_t *compressed_out);
sm_status sm_device_free(void *p);

/* Zeroes the accumulators and observation counts (enqueued on `stream`).
 * Errors: SM_ERR_INVALID_ARG (NULL mesh), SM_ERR_CUDA. */
sm_status sm_reset(sm_mesh *m, void *stream);

/* Copies the accumulators (n_x x c float32) and observation counts (n_x
 * uint32) to device buffers; either may be NULL.  With sm_load_state this
 * is the checkpoint / resume path: fusion is a sum over frames (Sec. 3.3.2),
 * so states of disjoint frame sets can be added. */
sm_status sm_read_state(sm_mesh *m, float *d_acc_out, uint32_t *d_cnt_out, void *stream);

/* Overwrites the accumulators and counts from device buffers (both required
 * when n_x > 0); a later render needs a new sm_normalise.
 * Errors (both state calls): SM_ERR_INVALID_ARG (NULL mesh, or NULL state
 * buffer for sm_load_state), SM_ERR_CUDA. */
sm_status sm_load_state(sm_mesh *m, const float *d_acc, const uint32_t *d_cnt, void *stream);

/* Synchronises `stream` and returns the first error a kernel latched since
 * the last sm_check (SM_ERR_INTERNAL), or SM_ERR_CUDA, or SM_OK.  Clears the
 * latch. */
sm_status sm_check(sm_mesh *m, void *stream);

/* Number of accumulator rows n_x (texels), or -1 for NULL. */
int64_t sm_num_rows(const sm_mesh *m);

/* Number of classes c, or -1 for NULL. */
int32_t sm_num_classes(const sm_mesh *m);

/* Releases the mesh and all library-owned device memory.  Synchronises the
 * device first.  NULL is a no-op. */
sm_status sm_mesh_free(sm_mesh *m);

/* Static description of a status code. */
const char *sm_status_string(sm_status s);

/* One-line detail of the calling thread's last failed call ("" if none). */
const char *sm_last_error(void);

/* Allocation-free rendering of row maps.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory, for
 * example a plugin whose host application owns every device allocation
 * through its own pool, or a latency-bound loop that must not call
 * cudaMalloc / cudaFree because they can block and synchronise the device.
 *
 * Renders N frames of a mesh given as plain arrays (no sm_mesh, no upload)
 * into d_idmap_out, N x H x W int32, with the same renderer as
 * sm_fuse_frames: every pixel gets the index of the triangle it sees (one row
 * per triangle, i.e. what sm_fuse_frames writes for a mesh uploaded without
 * texel steps), -1 for background.  Faces with an index outside [0, V) are
 * never drawn.  d_vertices V x 3 float32, d_faces F x 3 int32, d_K N
 * intrinsics and d_cam_to_world N x 16 float64 are device pointers.
 *
 * Scratch: the z-buffer of one frame and the N cameras live in a static
 * array of the library's device memory (SM_NOALLOC_MAX_PIXELS 64-bit keys +
 * SM_NOALLOC_MAX_FRAMES cameras, about 12 MiB), which every GPU that loads
 * the library holds until the process exits.  The call allocates nothing:
 * no cudaMalloc, cudaFree or allocating library routine.
 *   - The call runs on the device that holds d_idmap_out (made current for
 *     the call, then restored); the inputs must be memory of that device (or
 *     managed / mapped host memory it can address).  stream must belong to
 *     that device.
 *   - Each call looks up the array's device address on that device (no
 *     allocation).  The first call on a device may load the library's device
 *     code there: make it before any stream capture.
 *   - All calls share the array and it keeps the last call's contents (each
 *     call re-arms the z-buffer first).  Calls whose work overlaps on the GPU
 *     race on it: serialise them (one stream, or events).
 * Errors: SM_ERR_INVALID_ARG (NULL pointer, H x W > SM_NOALLOC_MAX_PIXELS,
 * N > SM_NOALLOC_MAX_FRAMES, V or F >= 2^31, an output that is not device
 * memory, an input on another device), SM_ERR_CUDA; all checks run before
 * anything is enqueued. */
#define SM_NOALLOC_MAX_PIXELS 1572864 /* 1.5 Mi pixels, e.g. 1296 x 968 */
#define SM_NOALLOC_MAX_FRAMES 1024
sm_status sm_render_rows_noalloc(const float *d_vertices, int64_t V, const int32_t *d_faces, int64_t F,
                                 const sm_intrinsics *d_K, const double *d_cam_to_world, int32_t N, int32_t H,
                                 int32_t W, int32_t *d_idmap_out, void *stream);

/* Kernel timing: when enabled, every launch of the kernels below is bracketed
 * by CUDA events on the launching stream (the raster kind brackets its two
 * kernels, cluster cull and raster, together).  Enabled or not, each such
 * launch is an NVTX range of the "labelfuse" domain named after its kind
 * ("project", "raster", ...), which profilers can show or filter on.  sm_profile_read synchronises
 * those events and returns the number of kernel launches and the total device
 * time since the last read (then clears them). */
typedef enum sm_kernel {
    SM_K_PROJECT = 0,   /* per-frame camera set-up (binary64)                  */
    SM_K_RASTER = 1,    /* triangle set-up, coverage and depth test            */
    SM_K_RESOLVE = 2,   /* z-buffer -> row map                                 */
    SM_K_COUNT = 3,     /* per-frame row histogram for w^(I)                   */
    SM_K_SCATTER = 4,   /* probability stream -> accumulator rows              */
    SM_K_NORMALISE = 5, /* rows -> distributions and labels                    */
    SM_K_RENDER = 6,    /* row maps -> label images                            */
    SM_K_QUEUE = 7,     /* raster + scatter of a whole call in the work queue  */
    SM_K_CONF = 8,      /* confidence weights inside sm_fuse_frames_confident  */
    SM_K_COUNT_KINDS = 9
} sm_kernel;

sm_status sm_profile_enable(sm_mesh *m, int32_t on);
sm_status sm_profile_read(sm_mesh *m, sm_kernel kernel, int64_t *launches, double *total_ms);

#ifdef __cplusplus
}
#endif

#endif /* LABELFUSE_H */
