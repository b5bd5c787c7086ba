/*
 * gsr.h -- C ABI of the GB300 2D-Gaussian surfel sensor renderer.
 *
 * The renderer rasterises 2D Gaussian surfels (arXiv 2503.11731, Sec. III-A,
 * "Unified Projection Scheme") into pinhole camera frames (RGB, expected
 * depth, normal) and spinning-LiDAR range images (range, intensity).  A frame
 * is produced by three calls that enqueue work on a caller stream:
 *
 *   gsr_preprocess   surfel -> per-(sensor, surfel) record, screen bound, tile count
 *   gsr_bin_sort     key duplication, on-device radix sort, tile ranges
 *   gsr_render_*     per-tile front-to-back compositing
 *
 * Conventions (all arrays row-major, float32 unless stated):
 *   world frame z up.  Camera frame x right, y down, z forward; LiDAR frame
 *   x forward, y left, z up.  world_to_sensor is a 4x4 rigid transform
 *   (rows [R|t; 0 0 0 1]).  Pixel (x, y) has centre (x + 0.5, y + 0.5).
 *   LiDAR row i (beam) has elevation el_max - i (el_max - el_min)/(beams-1);
 *   column j has azimuth az0 + (j + 0.5) 360/columns degrees.
 *
 * Memory: every pointer in a descriptor is DEVICE memory owned by the
 * caller, unless the field says "host".  The library allocates no device
 * memory: the caller allocates one workspace of gsr_workspace_size() bytes
 * (256-byte aligned) and passes it to every call of a frame.  `stream` is a
 * cudaStream_t (NULL = legacy default stream).  Calls are asynchronous;
 * argument errors are reported synchronously by the return code, device-side
 * conditions (key-capacity overflow, a bounded wait that gave up) are written
 * to a status word in the workspace and read with gsr_read_status().
 * No call traps or aborts; nothing crosses the ABI as an exception.
 */
#ifndef GSR_H
#define GSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GSR_MAX_SENSORS 16

typedef enum {
    GSR_OK = 0,
    GSR_ERR_INVALID_ARG = 1,  /* a null pointer, a bad size or an inconsistent descriptor */
    GSR_ERR_CUDA = 2,         /* a CUDA launch or query failed (see gsr_last_cuda_error)  */
    GSR_ERR_WORKSPACE = 3,    /* workspace too small or misaligned                        */
    GSR_ERR_CAPACITY = 4,     /* more tile/surfel pairs than max_dup (device status)      */
    GSR_ERR_TIMEOUT = 5,      /* a bounded device wait gave up (device status)            */
    GSR_ERR_UNSUPPORTED = 6,  /* e.g. SH degree > 3, a sensor kind not built              */
    GSR_ERR_TOO_LARGE = 7     /* a size beyond a fixed built-in limit                     */
} gsr_status;

typedef enum { GSR_SENSOR_PINHOLE = 0, GSR_SENSOR_LIDAR = 1, GSR_SENSOR_CYLINDRICAL = 2 } gsr_sensor_kind;

/*
 * Surfel table, structure of arrays, one row per surfel (Sec. III-A: the
 * 2DGS attributes {mu, R, S, rho, r, alpha}; colour from SH; r read as the
 * LiDAR intensity, rho as the LiDAR ray-drop probability).  Raw
 * (pre-activation) parameters:
 *   pos       [n][3]  centre mu (world)
 *   log_scale [n][2]  s_u = exp(.), s_v = exp(.)
 *   quat      [n][4]  (w, x, y, z), normalised by the renderer; R = [t_u t_v n]
 *   opacity   [n]     logit; o = sigmoid(.)
 *   sh        [n][(sh_degree+1)^2][3]  real SH coefficients (colour = max(0, SH + 0.5))
 *   intensity [n]     LiDAR intensity in [0,1] (may be NULL: 0)
 *   obj_id    [n]     int32 rigid-object index, -1 = background (may be NULL)
 *   ray_drop  [n]     LiDAR ray-drop logit; rho = sigmoid(.) (may be NULL: rho = 0)
 * All arrays 16-byte aligned.  `sees` says which sensors render the table:
 * GSR_SEES_CAMERAS | GSR_SEES_LIDARS (0 = all).  The paper reconstructs a
 * camera scene G^C and a separate LiDAR scene G^L (Sec. III-A); with `sees`
 * both share one plan, one sort and one compositing launch, each seen only
 * by its own sensors.
 */
#define GSR_SEES_CAMERAS 1 /* pinhole and cylindrical cameras */
#define GSR_SEES_LIDARS 2
typedef struct {
    int32_t n;
    int32_t sh_degree; /* 0..3 */
    const float* pos;
    const float* log_scale;
    const float* quat;
    const float* opacity;
    const float* sh;
    const float* intensity;
    const int32_t* obj_id;
    const float* ray_drop;
    int32_t sees;
} gsr_surfels;

/*
 * Rigid object poses (Sec. III-B, "Gaussian inplacing": a model matrix per
 * inserted actor): pose[k] = [R_o | t_o] row-major 3x4, DEVICE memory.
 * A surfel of object k renders with mu' = R_o mu + t_o, R' = R_o R; its SH
 * is evaluated at the view direction rotated back into the object frame.
 */
typedef struct {
    int32_t n_objects;
    const float* pose; /* [n_objects][12] */
} gsr_objects;

/*
 * Sensor descriptor (host memory).  Pinhole: Eq. 3 planes with the
 * intrinsics fx, fy, cx, cy.  LiDAR: Eq. 5 planes; width = azimuth columns,
 * height = beams.  Cylindrical (fisheye) camera, Eq. 4: pixel (x, y) looks
 * along azimuth phi = (x + 0.5 - cx)/fx about the camera's y axis at height
 * y_n = (y + 0.5 - cy)/fy on the unit cylinder, ray d = (sin phi, y_n,
 * cos phi); its planes are h_u = (cos phi, 0, -sin phi, 0) and, reading the
 * paper's pixel-frame h_v in the camera frame, h_v = (y_n sin phi, -1,
 * y_n cos phi, 0); depth = horizontal distance; the image must see azimuths
 * within [-pi, pi] (cx/fx and (width - cx)/fx at most pi).  Intersections
 * nearer than `near` (depth for the cameras, distance along the ray for
 * LiDAR) are rejected; surfels whose centre depth (range, horizontal
 * distance) is <= near are culled.
 */
typedef struct {
    int32_t kind;      /* gsr_sensor_kind */
    int32_t width;     /* pixels, or azimuth columns */
    int32_t height;    /* pixels, or beams (>= 2) */
    float fx, fy, cx, cy;
    float el_min_deg, el_max_deg, az0_deg;
    float near_plane;
    float world_to_sensor[16];
    float bg[3];       /* camera background, composited as bg * T */
    int32_t tile_w;    /* this sensor's screen tile (rays); 0 = the plan's tiling.  */
    int32_t tile_h;    /* w, h powers of two, w*h in {32,64,128,256}               */
    int32_t split_first; /* this sensor's list split (see gsr_tiling); 0 = the   */
    int32_t split_chunk; /* plan's                                               */
} gsr_sensor;

/* Default screen tiling of a plan's sensors (tile_w, tile_h powers of two,
 * tile_w * tile_h in {32,64,128,256}); a sensor may override it.
 * batch_depth = records staged in shared memory per step of a tile's walk
 * (double-buffered, 96 bytes each): 0 = the compositing CTA's thread count,
 * else one of 32, 64, 128, 256, 512.  It changes speed only, never results.
 * A tile list longer than split_first positions is split: its first
 * split_first positions are walked first, the rest in chunks of split_chunk
 * positions walked in parallel and merged in list order (0 = defaults 16384
 * and 384; split_first in [256, 2^24], split_chunk in [64, 2^24]).  The
 * merge reassociates products of transmittance, so results may change in
 * the last bits. */
typedef struct {
    int32_t tile_w, tile_h;
    int32_t batch_depth;
    int32_t split_first, split_chunk;
} gsr_tiling;

/*
 * A frame plan: sizes and the workspace layout, filled by gsr_plan_init()
 * on the host (no allocation).  Treat every field as read-only.
 */
typedef struct {
    int32_t n_surfels;
    int32_t n_sensors;
    gsr_sensor sensors[GSR_MAX_SENSORS];
    gsr_tiling tiling;
    int64_t max_dup;                      /* capacity of tile/surfel pairs        */
    int32_t tiles_x[GSR_MAX_SENSORS];
    int32_t tiles_y[GSR_MAX_SENSORS];
    int32_t tile_base[GSR_MAX_SENSORS + 1]; /* global tile id of each sensor's tile 0 */
    int32_t sort_ctas;                    /* persistent CTAs of the sort kernels  */
    uint64_t off[32];                     /* byte offsets of workspace regions    */
    uint64_t workspace_bytes;
} gsr_plan;

/*
 * Per-pixel outputs of a camera (DEVICE, planar [channel][H][W]; any may be
 * NULL to skip it).  With w_i = alpha_i T_i along the front-to-back order:
 *   rgb       [3][H][W]  sum w c + T bg
 *   depth     [H][W]     sum w z / sum w (0 where sum w == 0)
 *   normal    [3][H][W]  sum w n (camera frame, unnormalised)
 *   alpha     [H][W]     sum w
 *   trans     [H][W]     final transmittance T
 *   depth_acc [2][H][W]  sum w z, sum w z^2 (for the distortion loss)
 *   n_contrib [H][W]     uint32: list position of the last contributor + 1 (for the backward)
 *   n_walk    [H][W]     uint32: list entries the ray had to examine (its stop
 *                        position, or the whole tile list if it never saturated)
 */
typedef struct {
    float* rgb;
    float* depth;
    float* normal;
    float* alpha;
    float* trans;
    float* depth_acc;
    uint32_t* n_contrib;
    uint32_t* n_walk;
} gsr_camera_out;

/*
 * Per-ray outputs of a LiDAR (DEVICE, [beams][columns]; any may be NULL):
 *   range = sum w t / sum w (0 where sum w == 0), intensity = sum w r,
 *   alpha = sum w, trans = final T, n_contrib and n_walk as for the camera,
 *   ray_drop = sum w rho + T: the probability that the beam returns nothing
 *   (composited like the intensity; a beam that leaves the scene is dropped).
 */
typedef struct {
    float* range;
    float* intensity;
    float* alpha;
    float* trans;
    uint32_t* n_contrib;
    uint32_t* n_walk;
    float* ray_drop;
} gsr_lidar_out;

/*
 * Gradients of a loss w.r.t. one camera's per-pixel outputs (DEVICE,
 * planar, same shapes as gsr_camera_out; NULL = zero):
 *   rgb [3][H][W], alpha [H][W] (d/d sum w), depth_acc [2][H][W]
 *   (d/d sum w z, d/d sum w z^2), normal [3][H][W].
 */
typedef struct {
    float* rgb;
    float* alpha;
    float* depth_acc;
    float* normal;
} gsr_camera_grad;

/*
 * Gradients of a loss w.r.t. one LiDAR's per-ray outputs (DEVICE, planar,
 * [beams][columns] per plane; NULL = zero): intensity (d/d sum w r), alpha
 * (d/d sum w), depth_acc [2] (d/d sum w t, d/d sum w t^2; a loss on the
 * range B/A reaches A and B through these two), ray_drop
 * (d/d(sum w rho + T)).
 */
typedef struct {
    float* intensity;
    float* alpha;
    float* depth_acc;
    float* ray_drop;
} gsr_lidar_grad;

/* Gradients w.r.t. the raw surfel parameters (DEVICE, shapes of
 * gsr_surfels; accumulated with +=, so the caller zeroes them first). */
typedef struct {
    float* pos;
    float* log_scale;
    float* quat;
    float* opacity;
    float* sh;
    float* intensity; /* may be NULL */
    float* ray_drop;  /* may be NULL */
} gsr_surfel_grads;

/* Weights of the reconstruction loss (gsr_loss). */
typedef struct {
    float w_dist;      /* depth distortion weight (0.1)                  */
    float w_normal;    /* normal consistency weight (0.05)               */
    float mask_alpha;  /* normal term only where the 4 neighbours have sum w >= this (0.5) */
} gsr_loss_weights;

/* Weights of the LiDAR loss (gsr_lidar_loss). */
typedef struct {
    float w_range;      /* L1 range weight over returned rays (1.0)        */
    float w_intensity;  /* L1 intensity weight over returned rays (1.0)    */
    float w_drop;       /* ray-drop cross-entropy weight over all rays (0.1) */
} gsr_lidar_loss_weights;

/* ---------------------------------------------------------------- setup */

/* Fill `plan` for n_surfels surfels seen by n_sensors sensors (host only).
 * max_dup <= 0 picks a default capacity of 64 pairs per (sensor, surfel),
 * at most 2^31 - 1.  Errors: GSR_ERR_INVALID_ARG, GSR_ERR_UNSUPPORTED. */
gsr_status gsr_plan_init(gsr_plan* plan, int32_t n_surfels, const gsr_sensor* sensors,
                         int32_t n_sensors, const gsr_tiling* tiling, int64_t max_dup);

/* Bytes of device workspace the plan needs (host only). */
gsr_status gsr_workspace_size(const gsr_plan* plan, size_t* bytes);

/* ---------------------------------------------------------------- frame */

/*
 * Step (a), Eqs. 1-3 and 5 per (sensor, surfel): world->sensor transform,
 * near cull, the ray-to-(u,v) transform of Eq. 2 in closed form, the 3-sigma
 * screen (or angular) bound with the low-pass disc, the tile rectangle and
 * count, the SH colour and the facing normal.  Clears the status word.
 * `objects` may be NULL.
 */
gsr_status gsr_preprocess(const gsr_plan* plan, const gsr_surfels* surfels, const gsr_objects* objects,
                          void* workspace, size_t workspace_bytes, void* stream);

/*
 * gsr_preprocess for one part of the plan's surfels: table `surfels` (n
 * rows, its own SH degree) is surfels [first, first + n) of the plan, so a
 * frame can mix tables, e.g. a decoded SH-0 background and SH-3 posed
 * objects.  The status word is cleared only by the part with first == 0;
 * every plan surfel must be covered by exactly one part before
 * gsr_bin_sort.  Composite ties break by plan index as for one table.
 * Errors: GSR_ERR_INVALID_ARG when first < 0 or first + n > plan->n_surfels.
 */
gsr_status gsr_preprocess_part(const gsr_plan* plan, const gsr_surfels* surfels, const gsr_objects* objects,
                               int32_t first, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Step (b): compaction of visible records, radix sort of their centre-depth
 * keys, prefix sum of tile counts, key duplication (tile id, record), stable
 * radix sort by tile id -- together the stable sort of 64-bit (tile | depth)
 * keys -- and the [start, end) range of every tile.  More pairs than
 * max_dup sets GSR_ERR_CAPACITY in the status word (the excess is dropped).
 */
gsr_status gsr_bin_sort(const gsr_plan* plan, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Step (c): per-tile front-to-back compositing of camera `sensor`, pinhole
 * or cylindrical (Eq. 2 with the Eq. 3 or Eq. 4 planes: ray-splat (u,v),
 * low-pass fallback, alpha = min(0.99, o G), skip below 1/255, stop before
 * T (1 - alpha) < 1e-4).  Surfel batches are staged into shared memory by
 * bulk async copies.
 */
gsr_status gsr_render_camera(const gsr_plan* plan, const void* workspace, size_t workspace_bytes,
                             int32_t sensor, const gsr_camera_out* out, void* stream);

/* Step (c) for LiDAR `sensor` (Eq. 5 planes over the beam x azimuth tiling). */
gsr_status gsr_render_lidar(const gsr_plan* plan, const void* workspace, size_t workspace_bytes,
                            int32_t sensor, const gsr_lidar_out* out, void* stream);

/* -------------------------------------------------------------- training */

/*
 * Reconstruction loss of camera `sensor` against target_rgb [3][H][W]
 * (DEVICE), from the outputs of gsr_render_camera (fwd->rgb, alpha,
 * depth_acc, normal must be set), following the 2DGS regularisers the
 * paper's representation cites (Sec. II):
 *   L = mean|C - C*|                               (over 3 H W)
 *     + w_dist   * mean_px(A D - B^2)              A = sum w, B = sum w z, D = sum w z^2
 *     + w_normal * sum_px m (1 - N . N_d) / (H W)
 * N = sum w n; N_d = normalise(dY x dX) of the back-projected expected depth
 * B/A by central differences at the 4 neighbours; m = 1 on interior pixels
 * whose 4 neighbours have A >= mask_alpha and |dY x dX| > 0.  A pinhole
 * pixel back-projects to B/A ((x + 1/2 - cx)/fx, (y + 1/2 - cy)/fy, 1), a
 * cylindrical one (Eq. 4; its depth is the horizontal distance) to
 * B/A (sin phi, y_n, cos phi).
 * Writes loss[0..3] = (L, L1 term, distortion term, normal term) (DEVICE
 * float[4]) and the per-pixel gradients into *grad (all four planes
 * required; overwritten).  Uses workspace scratch; deterministic.  Pinhole
 * and cylindrical cameras; a LiDAR returns GSR_ERR_UNSUPPORTED (its loss is
 * gsr_lidar_loss).
 */
gsr_status gsr_loss(const gsr_plan* plan, void* workspace, size_t workspace_bytes, int32_t sensor,
                    const gsr_camera_out* fwd, const float* target_rgb, const gsr_loss_weights* weights,
                    float* loss, const gsr_camera_grad* grad, void* stream);

/*
 * Reverse-order backward rasteriser of camera `sensor` (pinhole or
 * cylindrical; a LiDAR returns GSR_ERR_UNSUPPORTED): each pixel walks its
 * tile list from its last contributor (fwd->n_contrib) back to the front,
 * recovering T_i = T_{i+1} / (1 - alpha_i) from the final T (fwd->trans;
 * no per-pixel lists are stored), and accumulates d(loss)/d(record) --
 * reduced over the warp before FP32 atomics -- into the workspace.
 * accumulate = 0 zeroes the record gradients first (first sensor of a step).
 * Must follow gsr_preprocess / gsr_bin_sort / gsr_render_camera (or
 * gsr_render_rig) of the same frame with the same workspace, that render
 * writing trans and n_contrib: the transmittance after each chunk of a
 * split tile list, where the backward walks of the other chunks start, is
 * kept in the workspace only by a render that writes trans.
 */
gsr_status gsr_backward_render(const gsr_plan* plan, void* workspace, size_t workspace_bytes, int32_t sensor,
                               const gsr_camera_out* fwd, const gsr_camera_grad* grad, int32_t accumulate,
                               void* stream);

/*
 * LiDAR loss of sensor `sensor` (GSR_SENSOR_LIDAR) against a recorded scan
 * (DEVICE [beams][columns]: target_range, 0 where the beam returned nothing;
 * target_intensity).  The paper reconstructs one LiDAR scene G^L apart from
 * the camera scenes (Sec. III-A, "Scene Reconstruction"), models the
 * ray-drop pattern (Sec. II, "Sensor Characteristics") and reports LiDAR
 * intensity quality and training speed (Sec. IV, the representation table)
 * without stating the loss; this one is
 *   L = w_range   * mean over returned rays |range - range*|
 *     + w_intensity * mean over returned rays |I - I*|
 *     + w_drop    * mean over all rays BCE(p, [range* == 0]),
 * p = ray_drop clamped to [2^-20, 1 - 2^-20] (no gradient where clamped),
 * range = B/A from gsr_render_lidar (no gradient where A = 0).  fwd->range,
 * alpha, intensity and ray_drop must be set.  Writes loss[0..3] = (L, range
 * term, intensity term, drop term) (DEVICE float[4]) and all four planes of
 * *grad (overwritten; depth_acc's second plane is 0).  Uses workspace
 * scratch; deterministic.  Another sensor kind returns GSR_ERR_UNSUPPORTED.
 */
gsr_status gsr_lidar_loss(const gsr_plan* plan, void* workspace, size_t workspace_bytes, int32_t sensor,
                          const gsr_lidar_out* fwd, const float* target_range, const float* target_intensity,
                          const gsr_lidar_loss_weights* weights, float* loss, const gsr_lidar_grad* grad,
                          void* stream);

/*
 * Reverse-order backward rasteriser of LiDAR `sensor` (Eq. 5 planes), as
 * gsr_backward_render: per-ray gradients *grad w.r.t. the composited
 * intensity, sum w, sum w t, sum w t^2 and ray drop (sum w rho + T, so the
 * drop's background is 1) reach each record's Q = adj(M), det(M), low-pass
 * centre, order key, opacity, intensity and rho.  fwd->trans and
 * fwd->n_contrib are required.  accumulate = 0 zeroes the record gradients
 * first.  Must follow gsr_preprocess / gsr_bin_sort / gsr_render_lidar (or
 * gsr_render_rig) of the same frame with the same workspace, that render
 * writing trans and n_contrib (as for gsr_backward_render).  Another
 * sensor kind returns GSR_ERR_UNSUPPORTED.
 */
gsr_status gsr_backward_render_lidar(const gsr_plan* plan, void* workspace, size_t workspace_bytes, int32_t sensor,
                                     const gsr_lidar_out* fwd, const gsr_lidar_grad* grad, int32_t accumulate,
                                     void* stream);

/*
 * Chain the record gradients of all sensors back to the raw surfel
 * parameters (pos, log_scale, quat, opacity logit, SH, incl. the view
 * direction of the SH colour; for LiDAR records also intensity and the
 * ray-drop logit, out->intensity / out->ray_drop when not NULL),
 * accumulating into *out.  Every sensor model: pinhole (Eq. 3 Jacobian),
 * cylindrical and LiDAR (the adjugate of M = [a b ms] and the centre's
 * angles).
 */
gsr_status gsr_backward_preprocess(const gsr_plan* plan, const void* workspace, size_t workspace_bytes,
                                   const gsr_surfels* surfels, const gsr_objects* objects,
                                   const gsr_surfel_grads* out, void* stream);

/*
 * gsr_loss_noalloc -- the same loss and per-pixel gradients as gsr_loss, for
 * callers that cannot allocate device memory: code that runs where
 * cudaMalloc is off limits (inside a caller's own memory pool or arena, in a
 * process whose allocator is owned by another runtime, or on a path that must
 * never grow the device footprint) and so cannot provide a plan workspace.
 * The paper has no counterpart; this is an interface convenience.
 *
 * It takes no plan and no workspace.  Its scratch (6 floats per pixel plus
 * block partial sums) lives in one fixed array in the library's own device
 * memory, sized for GSR_NOALLOC_MAX_PIXELS pixels (48 MiB + 96 KiB); every
 * GPU that loads the library holds that array until the process exits.
 * camera: the pinhole or cylindrical descriptor (host); fwd->rgb, alpha, depth_acc, normal,
 * target_rgb, loss[4] and all four planes of *grad as for gsr_loss.
 * Errors: GSR_ERR_TOO_LARGE if width * height > GSR_NOALLOC_MAX_PIXELS;
 * GSR_ERR_INVALID_ARG / GSR_ERR_UNSUPPORTED as for gsr_loss.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current): make that first call before any stream
 * capture.  No call allocates or frees device memory.  All calls share the
 * one array, so calls that overlap on the GPU (on different streams, or from
 * different threads, on the same device) race and must be serialised by the
 * caller; nothing in the array needs to start at zero.
 */
#define GSR_NOALLOC_MAX_PIXELS 2097152
gsr_status gsr_loss_noalloc(const gsr_sensor* camera, const gsr_camera_out* fwd, const float* target_rgb,
                            const gsr_loss_weights* weights, float* loss, const gsr_camera_grad* grad,
                            void* stream);

/* gsr_backward_render (accumulate = 0) + gsr_backward_preprocess for one camera. */
gsr_status gsr_backward(const gsr_plan* plan, void* workspace, size_t workspace_bytes, int32_t sensor,
                        const gsr_camera_out* fwd, const gsr_camera_grad* grad, const gsr_surfels* surfels,
                        const gsr_objects* objects, const gsr_surfel_grads* out, void* stream);

/* -------------------------------------------------------- learned decode */

/*
 * Anchors of a neural-Gaussian scene (Sec. III-A, "Scene Reconstruction":
 * anchors organised as in Scaffold-GS; an MLP infers the 2DGS attributes of
 * each anchor's k offset surfels).  DEVICE arrays:
 *   pos [n][3], feature [n][feat_dim], scale [n] (l_a > 0), offsets [n][k][3],
 *   intensity [n][k] (LiDAR intensity of each offset surfel; may be NULL).
 * Built shapes: k = 10, feat_dim = 32 (others return GSR_ERR_UNSUPPORTED).
 */
typedef struct {
    int32_t n;
    int32_t k;
    int32_t feat_dim;
    const float* pos;
    const float* feature;
    const float* scale;
    const float* offsets;
    const float* intensity;
} gsr_anchors;

/* The decode MLP, FP32 masters (DEVICE, row-major): w1 [feat_dim+4][hidden],
 * b1 [hidden], w2 [hidden][10 k], b2 [10 k]; hidden = 64.  head: what the
 * 10 outputs of an offset mean (see gsr_decode_anchors). */
#define GSR_HEAD_CAMERA 0 /* the camera scene G^C */
#define GSR_HEAD_LIDAR 1  /* the LiDAR scene G^L   */
typedef struct {
    int32_t hidden;
    const float* w1;
    const float* b1;
    const float* w2;
    const float* b2;
    int32_t head;
} gsr_mlp;

/* Gradients of the MLP (and optionally of the anchor features), accumulated (+=). */
typedef struct {
    float* w1;
    float* b1;
    float* w2;
    float* b2;
    float* feature; /* [n][feat_dim], may be NULL */
} gsr_mlp_grads;

/* A writable surfel table (DEVICE) with degree-0 SH, as produced by the decode:
 * pos [N][3], log_scale [N][2], quat [N][4], opacity [N], sh [N][1][3], intensity [N]
 * (may be NULL), ray_drop [N] (LiDAR head; may be NULL). */
typedef struct {
    float* pos;
    float* log_scale;
    float* quat;
    float* opacity;
    float* sh;
    float* intensity;
    float* ray_drop;
} gsr_surfel_table;

#define GSR_DECODE_BF16_TENSOR 0 /* BF16 inputs/weights on tcgen05 tensor cores, FP32 accumulation */
#define GSR_DECODE_F32 1         /* FP32 on the SIMT cores (reference path)                      */

/*
 * Decode every anchor into k surfels (surfel a k + j = offset j of anchor a):
 *   X = [feature, (x_a - o)/|x_a - o|, |x_a - o|], H = ReLU(X w1 + b1),
 *   y = H w2 + b2; offset j: opacity logit y0, log-scale y4..5 + ln l_a, raw
 *   quaternion y6..9, centre x_a + l_a offset_j, and
 *     camera head: colour sigmoid(y1..3) stored as degree-0 SH (out->sh
 *                  required), intensity from the anchors;
 *     LiDAR head:  intensity sigmoid(y1), ray-drop logit y2 (y3 unused),
 *                  SH written as 0 when out->sh is set (the LiDAR scene has
 *                  no colour).
 * origin (host float[3]) is the view origin o (camera centre; rig centre for
 * a rig).  cull_camera (host, may be NULL): anchors whose sphere of radius
 * l_a max|offset| + 3 m is outside that pinhole's frustum get opacity logit
 * -1e4.  device_status (DEVICE uint32, may be NULL) records GSR_ERR_TIMEOUT
 * if a bounded wait on the tensor cores gave up.
 */
gsr_status gsr_decode_anchors(const gsr_anchors* anchors, const gsr_mlp* mlp, const float* origin,
                              const gsr_sensor* cull_camera, int32_t precision, const gsr_surfel_table* out,
                              uint32_t* device_status, void* stream);

/*
 * Back-propagate d(loss)/d(decoded surfel table) (opacity, log_scale, quat,
 * and sh for the camera head or intensity and ray_drop for the LiDAR head,
 * of the table produced by gsr_decode_anchors with the same arguments)
 * through the decode activations and the MLP (FP32), accumulating into *out.
 */
gsr_status gsr_decode_backward(const gsr_anchors* anchors, const gsr_mlp* mlp, const float* origin,
                               const gsr_sensor* cull_camera, const gsr_surfel_grads* d_surfels,
                               const gsr_mlp_grads* out, void* stream);

/* Adam step on an FP32 master array (step counts from 1; bias-corrected). */
gsr_status gsr_adam(float* param, const float* grad, float* m, float* v, int64_t n, float lr, float beta1,
                    float beta2, float eps, int32_t step, void* stream);

/* ------------------------------------------------------------ whole rig */

/*
 * Step (c) for every sensor of the plan -- a surround rig of cameras and
 * LiDARs of mixed resolutions -- in ONE persistent launch: resident CTAs
 * pull (sensor, tile) items from a work queue ordered longest list first
 * (built by gsr_bin_sort) and composite each with the camera or LiDAR rules.
 * camera_outs and lidar_outs are host arrays of plan->n_sensors entries
 * indexed by sensor: entry i of camera_outs is used when sensor i is a
 * pinhole, entry i of lidar_outs when it is a LiDAR (an array may be NULL if
 * the plan has no sensor of that kind).  Results equal gsr_render_camera /
 * gsr_render_lidar per sensor.
 */
gsr_status gsr_render_rig(const gsr_plan* plan, const void* workspace, size_t workspace_bytes,
                          const gsr_camera_out* camera_outs, const gsr_lidar_out* lidar_outs, void* stream);

/*
 * A frame -- gsr_preprocess, gsr_bin_sort, gsr_render_rig, or the subset
 * selected by `stages` (bit 0 preprocess, bit 1 bin_sort, bit 2 render_rig;
 * 7 = the whole frame) -- captured once into a CUDA graph on `stream` (a
 * created stream, not the legacy default one) and replayed with
 * gsr_frame_graph_launch.  The graph keeps every pointer it was created
 * with: update the surfel table, object poses and outputs in place between
 * launches.  The handle is host memory owned by the library until
 * gsr_frame_graph_destroy.
 */
#define GSR_STAGE_PREPROCESS 1
#define GSR_STAGE_BIN_SORT 2
#define GSR_STAGE_RENDER_RIG 4
typedef struct gsr_frame_graph_s gsr_frame_graph;
gsr_status gsr_frame_graph_create(const gsr_plan* plan, const gsr_surfels* surfels, const gsr_objects* objects,
                                  void* workspace, size_t workspace_bytes, const gsr_camera_out* camera_outs,
                                  const gsr_lidar_out* lidar_outs, int32_t stages, void* stream,
                                  gsr_frame_graph** graph);
gsr_status gsr_frame_graph_launch(gsr_frame_graph* graph, void* stream);
gsr_status gsr_frame_graph_destroy(gsr_frame_graph* graph);

/*
 * Copy the device status word to the host (synchronises `stream`).
 * *device_status receives GSR_OK, GSR_ERR_CAPACITY or GSR_ERR_TIMEOUT;
 * *n_visible and *n_pairs (may be NULL) the visible records and tile/surfel
 * pairs of the last gsr_bin_sort.
 */
gsr_status gsr_read_status(const gsr_plan* plan, const void* workspace, int32_t* device_status,
                           int64_t* n_visible, int64_t* n_pairs, void* stream);

/*
 * Measurement kernel of the compositing roofline (no counterpart in the
 * paper): `blocks` CTAs of 256 threads, each thread running 8 independent
 * FP32 fused multiply-add chains of `iters` steps, the sums written to
 * out[blocks * 256] (device memory, caller-owned).  *fmas receives the
 * multiply-adds launched; the caller times the launch on `stream` with its
 * own events, which gives the GPU's FP32 FMA issue rate.  Async.
 * Errors: GSR_ERR_INVALID_ARG (null pointer, blocks or iters <= 0),
 * GSR_ERR_CUDA (launch failure).
 */
gsr_status gsr_fma_peak_kernel(float* out, int32_t blocks, int32_t iters, int64_t* fmas, void* stream);

/*
 * Self-test of the device-side give-up path (no counterpart in the paper:
 * the bounded waits are this library's, not the method's).  Launches one
 * CTA that arms an mbarrier for 16 bytes no copy will deliver and waits on
 * it with the library's bounded wait, `tries` tries (1 .. 2^20); the wait
 * gives up, the kernel records GSR_ERR_TIMEOUT in the plan's status word
 * (read it with gsr_read_status) and returns.  No copy or tensor-core
 * operation is outstanding at any point, so the context stays usable; the
 * next gsr_preprocess(_part) with first == 0 clears the status word.
 * Async on `stream`; the workspace is the plan's (256-byte aligned).
 * Errors: GSR_ERR_INVALID_ARG (null pointer, tries out of range),
 * GSR_ERR_WORKSPACE, GSR_ERR_CUDA (launch failure).
 */
gsr_status gsr_selftest_wait_timeout(const gsr_plan* plan, void* workspace, size_t workspace_bytes, uint32_t tries,
                                     void* stream);

/* ------------------------------------------------------------- autotune */

/*
 * Search space of gsr_autotune (host memory).  Every camera takes the same
 * camera tile, every LiDAR the same LiDAR tile; split_firsts / split_chunks
 * are the plan's list split (the cameras'), lidar_split_* the LiDARs' own
 * (gsr_sensor.split_*; their long horizon lists favour shorter first
 * walks); n_* = 0 keeps the plan's choice.  Tiles obey gsr_tiling's rule;
 * batch depths and split lengths are values gsr_tiling accepts.  Each
 * candidate renders `warmup` untimed and `reps` timed frames (reps >= 1).
 */
#define GSR_AUTOTUNE_MAX 8
typedef struct {
    int32_t n_camera_tiles;
    int32_t camera_tiles[GSR_AUTOTUNE_MAX][2];
    int32_t n_lidar_tiles;
    int32_t lidar_tiles[GSR_AUTOTUNE_MAX][2];
    int32_t n_batch_depths;
    int32_t batch_depths[GSR_AUTOTUNE_MAX];
    int32_t n_split_firsts;
    int32_t split_firsts[GSR_AUTOTUNE_MAX];
    int32_t n_split_chunks;
    int32_t split_chunks[GSR_AUTOTUNE_MAX];
    int32_t n_lidar_split_firsts;
    int32_t lidar_split_firsts[GSR_AUTOTUNE_MAX];
    int32_t n_lidar_split_chunks;
    int32_t lidar_split_chunks[GSR_AUTOTUNE_MAX];
    int32_t warmup, reps;
} gsr_autotune_space;

/* One measured candidate: ms = mean frame time (preprocess + bin_sort +
 * render_rig), or a negative value when the candidate's frame failed (e.g.
 * the pair capacity of its plan overflowed).  lidar_tile is the first
 * LiDAR's tile, lidar_tiles the tiles of the plan's first
 * GSR_AUTOTUNE_LIDARS LiDARs in plan order (later LiDARs take the last). */
#define GSR_AUTOTUNE_LIDARS 4
typedef struct {
    int32_t camera_tile[2];
    int32_t lidar_tile[2];
    int32_t batch_depth;
    int32_t split_first, split_chunk;
    int32_t lidar_split_first, lidar_split_chunk; /* 0 = the plan's */
    int32_t lidar_tiles[GSR_AUTOTUNE_LIDARS][2];
    float ms;
} gsr_autotune_trial;

typedef struct {
    gsr_plan plan;        /* the input plan re-initialised with the fastest tiling */
    float best_ms;
    int32_t n_tried;
    gsr_autotune_trial tried[(7 + GSR_AUTOTUNE_LIDARS) * GSR_AUTOTUNE_MAX + 1];
} gsr_autotune_result;

/* Workspace bytes gsr_autotune needs: the largest over the candidates
 * (host only). */
gsr_status gsr_autotune_workspace_size(const gsr_plan* plan, const gsr_autotune_space* space, size_t* bytes);

/*
 * Autotuner of the batched rig frame (the paper prescribes none; tile shape,
 * staging depth and list splitting are this implementation's free
 * parameters).  Coordinate descent from the plan's tiling: the camera tile
 * over its candidates, then one LiDAR tile for every LiDAR, then each of the
 * first GSR_AUTOTUNE_LIDARS LiDARs' tile on its own (a 32-beam and a 128-beam
 * LiDAR favour different shapes), the batch depth, the first split length
 * and the later chunk length, then the LiDARs' two split lengths,
 * each candidate timed with CUDA
 * events over whole frames of the given surfels: `parts` (n_parts tables,
 * consecutive in the plan from surfel 0, as gsr_preprocess_part) and
 * `objects` (may be NULL), rendered into camera_outs / lidar_outs (as
 * gsr_render_rig).  Synchronous: it waits for `stream` and leaves the last
 * candidate's frame in the outputs.  Results never depend on the choice
 * (only lists and staging do).  Errors: GSR_ERR_INVALID_ARG,
 * GSR_ERR_WORKSPACE (workspace smaller than gsr_autotune_workspace_size),
 * GSR_ERR_CUDA.
 */
gsr_status gsr_autotune(const gsr_plan* plan, const gsr_surfels* parts, int32_t n_parts,
                        const gsr_objects* objects, const gsr_autotune_space* space, void* workspace,
                        size_t workspace_bytes, const gsr_camera_out* camera_outs,
                        const gsr_lidar_out* lidar_outs, gsr_autotune_result* result, void* stream);

/* Readable name of a status code (static storage). */
const char* gsr_status_string(gsr_status s);

/* The last CUDA error string seen by this thread's calls ("" if none). */
const char* gsr_last_cuda_error(void);

/*
 * sizeof of the ABI structs, for bindings that mirror them (host only):
 * which = 0 gsr_plan, 1 gsr_sensor, 2 gsr_surfels, 3 gsr_objects,
 * 4 gsr_camera_out, 5 gsr_lidar_out, 6 gsr_tiling, 7 gsr_camera_grad,
 * 8 gsr_surfel_grads, 9 gsr_loss_weights, 10 gsr_anchors, 11 gsr_mlp,
 * 12 gsr_mlp_grads, 13 gsr_surfel_table, 14 gsr_autotune_space,
 * 15 gsr_autotune_result, 16 gsr_zone_grid, 17 gsr_streamer,
 * 18 gsr_lidar_grad, 19 gsr_lidar_loss_weights.  Returns 0 for other values.
 */
size_t gsr_struct_size(int32_t which);

/* ------------------------------------------------ large-scale streaming */

/*
 * Zones of a large scene (Sec. III-A, "Support Large-scale Scenes": frames
 * are clustered by their XY location into 40 x 40 m zones with 25 % relative
 * padding, and while rendering two threads double-buffer the zones, swapping
 * in the Gaussians of the next block as the vehicle moves between blocks).
 * Zone (i, j), 0 <= i < nx, 0 <= j < ny, id j nx + i, is the square
 * [x0 + i s, x0 + (i+1) s) x [y0 + j s, y0 + (j+1) s), s = zone_size; its
 * surfels are those whose centre lies in the square grown by padding x s
 * on every side (padding in [0, 0.5]: a surfel belongs to up to four
 * zones).  Bounds are compared in double precision.  Host memory, host only.
 */
typedef struct {
    float x0, y0;
    float zone_size;
    float padding;
    int32_t nx, ny;
} gsr_zone_grid;

/* Zone whose unpadded square holds (x, y), or -1 outside the grid (or for a bad grid). */
int32_t gsr_zone_of(const gsr_zone_grid* grid, float x, float y);

/* counts[z] = surfels of zone z (pos: HOST [n][3] world centres). */
gsr_status gsr_zone_count(const gsr_zone_grid* grid, const float* pos, int64_t n, int64_t* counts);

/* Members in CSR form: offsets [nx ny + 1] = exclusive prefix of the counts,
 * members[offsets[z] .. offsets[z+1]) = ascending surfel indices of zone z.
 * GSR_ERR_INVALID_ARG if the offsets do not fit the table's counts. */
gsr_status gsr_zone_members(const gsr_zone_grid* grid, const float* pos, int64_t n, const int64_t* offsets,
                            int64_t* members);

/* Gather surfels members[0 .. count) of a HOST table into contiguous HOST
 * arrays `out` (sized for count; intensity and ray_drop written when `out`
 * has them: 0 / -1e4 where the table has none).  Zones are packed once, so
 * a swap is one copy per array. */
gsr_status gsr_zone_pack(const gsr_surfels* table, const int64_t* members, int64_t count,
                         const gsr_surfel_table* out);

/*
 * Double-buffered zone streamer.  The caller allocates the struct and two
 * DEVICE tables of `capacity` surfels (its SH degree), and owns the copy
 * stream; the library creates two CUDA events per buffer (released by
 * gsr_streamer_destroy) and allocates no memory.
 *   prefetch(zone, host_zone): unless the zone is already in a buffer, copy
 *     its packed arrays (HOST, pinned for the copy to overlap) into the back
 *     buffer on the copy stream -- after the render stream has released that
 *     buffer -- and mark the slots beyond its surfels culled (opacity logit
 *     -1e4).  GSR_ERR_CAPACITY if the zone is larger than a buffer.
 *   acquire(zone, render_stream, out): make the zone's buffer the front
 *     (swapping if it is the back one), make render_stream wait for its
 *     copy, and describe it in *out (n = capacity; the plan renders
 *     `capacity` surfels).  GSR_ERR_INVALID_ARG if the zone was never
 *     prefetched.
 * Treat every field as read-only.
 */
typedef struct {
    int32_t capacity;
    int32_t sh_degree;
    gsr_surfel_table buf[2]; /* DEVICE */
    int32_t zone[2];         /* zone held by each buffer, -1 = none */
    int32_t count[2];        /* its surfels */
    int32_t front;           /* buffer frames draw from */
    int32_t released_valid[2];
    void* copy_stream;
    void* ready[2];          /* cudaEvent_t: the buffer's copy is done */
    void* released[2];       /* cudaEvent_t: the render stream is done with the buffer */
} gsr_streamer;

gsr_status gsr_streamer_init(gsr_streamer* s, int32_t capacity, int32_t sh_degree, const gsr_surfel_table* buffers,
                             void* copy_stream);
gsr_status gsr_streamer_prefetch(gsr_streamer* s, int32_t zone, const gsr_surfels* host_zone);
gsr_status gsr_streamer_acquire(gsr_streamer* s, int32_t zone, void* render_stream, gsr_surfels* out);
gsr_status gsr_streamer_destroy(gsr_streamer* s);

/* ------------------------------------------------- workspace inspection */

/*
 * Device pointers into the workspace, for tests and tools (no copy):
 * which = 0 records (float4 x 6 per (sensor, surfel) slot), 1 tile rects
 * (ushort4 per slot: tx0, tx1, ty0, ty1; tx1 may exceed tiles_x - 1 for a
 * LiDAR azimuth wrap), 2 tile counts (uint32 per slot), 3 depth keys
 * (float bits per slot), 4 sorted pair tile ids (uint32), 5 sorted pair
 * slots (uint32), 6 tile ranges (uint2 per global tile), 7 visible slots in
 * depth order (uint32), 8 list splits (uint4 per global tile: x = chunks
 * after the first, 0 = not split).
 */
gsr_status gsr_workspace_region(const gsr_plan* plan, const void* workspace, int32_t which, void** ptr,
                                size_t* bytes);

#ifdef __cplusplus
}
#endif

#endif /* GSR_H */
