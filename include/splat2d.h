/*
 * splat2d.h -- C ABI of the GB300 (sm_103a) differentiable 2D Gaussian surfel
 * rasterizer: the data-parallel hot path of Flash-Mono's mapping backend.
 *
 * What is rendered (Sec. 3, Eq. 1 and the 2DGS surfel primitive it adopts):
 * each surfel i has a center mu_i, colour c_i, opacity sigma_i, rotation r_i
 * (a quaternion) and two tangent scales s_i.  Seen from a pinhole camera
 * (intrinsics fx, fy, cx, cy; world-to-camera pose [R|t]) the ray through a
 * pixel meets the surfel plane at local coordinates (u, v) (ray-splat
 * intersection); the surfel's weight there is
 *     w_i = min(alpha_max, sigma_i * max(exp(-(u^2+v^2)/2),
 *                                        exp(-|x - c_i|^2 / (2 lowpass^2))))
 * (object-space / screen-space low-pass max, c_i the projected center), and
 * the pixel's colour, depth and accumulated alpha are, front to back in
 * depth order,
 *     (I, D, A) = sum_i (c_i, z_i, 1) w_i prod_{j<i} (1 - w_j)     (Eq. 1)
 * with z_i the depth of the surfel center along the optical axis, plus a
 * camera-frame normal N = sum_i n_i w_i prod_{j<i}(1 - w_j).  Pairs with
 * w_i < alpha_min are skipped, and a pixel stops before the first surfel that
 * would take its transmittance below t_min.  I also gets T_final * bg.
 *
 * The backward pass gives dL/d(means, scales, quats, opacity, rgb) and, per
 * view, dL/dxi for the left perturbation T_cw <- Exp(xi) T_cw, xi = (rho,
 * phi), evaluated at xi = 0 (the camera se(3) tangent used when refining
 * poses).
 *
 * Conventions for every call:
 *  - Host pointers: the splat2d_config, splat2d_problem (and its view array),
 *    splat2d_surfels and splat2d_grads structs themselves.  Device pointers:
 *    the arrays they point to, the workspace and every image buffer.
 *  - The caller owns all memory.  The library never allocates device memory:
 *    the caller allocates a workspace of splat2d_workspace_size() bytes
 *    (256-byte aligned), zero-fills it once before its first use, and passes
 *    the same problem to every call.  (The gradient records in the workspace
 *    are accumulated by the tile adjoint and cleared again by the chain rule,
 *    so they stay zero between iterations.)
 *  - Calls are asynchronous on `stream`, make no host synchronisation and no
 *    allocation, and are capturable in a CUDA graph (except
 *    splat2d_status / splat2d_stats, which synchronise).
 *  - Return value: SPLAT2D_OK or a negative error code for a problem found on
 *    the host (bad argument, workspace too small, CUDA launch error).
 *    Conditions found on the device (instance capacity exceeded, a bounded
 *    wait that gave up) are recorded in the workspace and read with
 *    splat2d_status() after the stream is synchronised.
 *  - Layouts: FP32 everywhere.  Surfel arrays are row-major [N, k].  Images
 *    are planar and packed per view: view v's RGB and normal occupy
 *    [3][H_v][W_v] at element offset 3*pixel_offset_v of their buffers, and
 *    its depth and alpha occupy [H_v][W_v] at pixel_offset_v.  Pixel (i, j)
 *    is sampled at (i + 0.5, j + 0.5).
 */
#ifndef SPLAT2D_H
#define SPLAT2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (0 = legacy default stream). */
typedef struct CUstream_st* splat2d_stream;

enum {
  SPLAT2D_OK = 0,
  SPLAT2D_ERR_INVALID_ARG = -1,        /* a host-side argument is out of range */
  SPLAT2D_ERR_WORKSPACE_TOO_SMALL = -2,
  SPLAT2D_ERR_CUDA = -3,               /* a CUDA launch or copy failed */
  SPLAT2D_ERR_CAPACITY = -4,           /* device: more tile instances than instance_capacity */
  SPLAT2D_ERR_TIMEOUT = -5,            /* device: a bounded wait gave up */
  SPLAT2D_ERR_NO_DEVICE = -6,
  SPLAT2D_ERR_BOUNDS = -7              /* device, checked builds only: an index check failed and the access was skipped */
};

/* One camera and the surfel range it renders. */
typedef struct {
  int32_t width, height;        /* pixels, 1..32768 */
  float fx, fy, cx, cy;         /* pinhole intrinsics, pixels */
  float Rt[12];                 /* world -> camera [R | t], row-major 3x4 */
  int64_t surfel_offset;        /* first surfel of the range this view renders */
  int64_t surfel_count;         /* number of surfels in the range */
  int64_t pixel_offset;         /* start of this view's pixels in the packed images */
} splat2d_view;

/* Surfel parameters (device arrays, FP32, row-major). */
typedef struct {
  const float* means;    /* [N, 3] world centers */
  const float* scales;   /* [N, 2] tangent scales (linear) */
  const float* quats;    /* [N, 4] rotation (w, x, y, z), any nonzero norm: normalised inside */
  const float* opacity;  /* [N] in [0, 1] (linear) */
  const float* rgb;      /* [N, 3] colour */
  int64_t n;
} splat2d_surfels;

/* Writable surfel arrays (device, FP32, row-major), for the map-maintenance
 * calls that produce or update surfels in place. */
typedef struct {
  float* means;    /* [N, 3] */
  float* scales;   /* [N, 2] */
  float* quats;    /* [N, 4] (w, x, y, z) */
  float* opacity;  /* [N] */
  float* rgb;      /* [N, 3] */
} splat2d_surfel_buffers;

/* Gradient outputs (device arrays).  Accumulated into (+=): zero them first.
 * Any pointer may be NULL to skip that output. */
typedef struct {
  float* means;    /* [N, 3] */
  float* scales;   /* [N, 2] */
  float* quats;    /* [N, 4] */
  float* opacity;  /* [N] */
  float* rgb;      /* [N, 3] */
  float* pose;     /* [n_views, 6]: dL/d(rho_xyz, phi_xyz) */
} splat2d_grads;

/* Rasterizer constants.  Defaults (splat2d_default_config): 8x8 tiles,
 * chunk 128 (forward) and 64 (backward), alpha in [1/255, 0.99], t_min 1e-4,
 * lowpass sqrt(1/2) px, z_near 0.01, black background. */
typedef struct {
  int32_t tile_w, tile_h;   /* one of 8x8, 16x16, 32x8 */
  int32_t chunk;            /* surfels staged per shared-memory batch: 64, 128, 256 (or 512 with 256-pixel tiles) */
  float alpha_min;          /* skip pairs with alpha below this */
  float alpha_max;          /* clamp of alpha (keeps the reverse pass finite) */
  float t_min;              /* stop a pixel before T would drop below this */
  float lowpass_sigma;      /* screen-space low-pass std-dev in pixels (0 = off) */
  float z_near;             /* cull surfels whose opacity-aware disk reaches z <= z_near */
  float bg[3];              /* background colour added as T_final * bg */
  uint32_t flags;           /* SPLAT2D_FLAG_* */
  int32_t bwd_chunk;        /* chunk of the backward compositing pass (0 = chunk; same values as chunk) */
} splat2d_config;

/* flags */
#define SPLAT2D_FLAG_NO_STATS 1u   /* skip the pair counters (kept by default) */
/* Depth output per pixel from the ray-splat intersection: each pair
 * contributes the depth of the point where the pixel's ray meets the surfel
 * plane (2D Gaussian Splatting's per-pixel geometry) wherever the
 * object-space term of the low-pass max decides, and its center's depth
 * z_i elsewhere.  Default off: z_i of the center for every pair, as Eq. 1
 * of the paper (Sec. 3) writes it. */
#define SPLAT2D_FLAG_DEPTH_RAY 2u
/* Bits 8..15 of flags: forward tail threshold, pixels per warp of a tile below
 * which the forward shares the tile's remaining pixels across all warps
 * (0 = the default of 6; 255 = always).  A launch-shape knob for the
 * autotuner: it changes the schedule, not the result beyond rounding. */
#define SPLAT2D_FLAG_TAIL_SHIFT 8

/* The shape of one problem: the views (host array) and sizes.  Pass the same
 * problem (same values) to every call that uses one workspace. */
typedef struct {
  const splat2d_view* views;   /* host array of n_views */
  int32_t n_views;             /* 1..4096 */
  int64_t n_surfels;           /* size of the surfel arrays */
  int64_t instance_capacity;   /* max (tile, surfel) instances per iteration */
} splat2d_problem;

/* Device-side counters of the last iteration (see splat2d_stats). */
typedef struct {
  int64_t status;              /* SPLAT2D_OK or a device error code */
  int64_t needed_capacity;     /* instances the last binning needed */
  int64_t n_instances;         /* instances binned and sorted */
  int64_t n_visible;           /* visible (view, surfel) pairs */
  int64_t fwd_pairs_evaluated; /* (pixel, surfel) pairs whose alpha the forward computed */
  int64_t fwd_pairs_blended;   /* ... of which blended */
  int64_t bwd_pairs_evaluated; /* (pixel, surfel) pairs the reverse pass recomputed */
  int64_t bwd_pairs_blended;   /* ... of which carried gradient */
  int64_t sort_passes;         /* radix passes run */
  int64_t bwd_terms_outside;   /* gradient terms outside their chunk's fixed-point range, added in float */
  int64_t reserved[6];
} splat2d_stats_t;

/* Fill `cfg` with the defaults above. */
void splat2d_default_config(splat2d_config* cfg);

/* Bytes of workspace the problem needs (0 if the arguments are invalid).
 * The workspace holds, per (view, surfel) pair of every view's range, an
 * 80-byte render record, an 80-byte gradient record, a 4-byte tile count
 * and a 16-byte binning entry (depth key, pixel rect, tile count);
 * per unit of instance_capacity, 24 bytes of sort keys and values, an 80-byte
 * sorted-order record copy and tile_w * tile_h / 8 bytes of blended-pair
 * masks; and 12 bytes per pixel. */
size_t splat2d_workspace_size(const splat2d_config* cfg, const splat2d_problem* prob);

/*
 * Follows: Sec. 3 ("Preliminaries"), the 2DGS surfel the paper adopts
 * (position, colour, opacity, rotation, 2D scale) and the per-surfel terms
 * of Eq. 1 (the weight w_i of a pixel, the depth z_i along the optical
 * axis); the extent is the support of w_i >= alpha_min.
 *
 * Per-surfel preprocess (one launch over every view's surfel range): camera
 * transform, tangent frame from the normalised quaternion, the ray-splat
 * intersection transform, projected center, depth key, camera normal turned
 * to face the camera, culls, and the opacity-aware screen extent united with
 * the low-pass square, as a pixel rect.  Writes render records into `ws` and
 * resets the device status.  Returns SPLAT2D_ERR_INVALID_ARG for a bad
 * problem or surfel count mismatch, SPLAT2D_ERR_WORKSPACE_TOO_SMALL if
 * ws_bytes < splat2d_workspace_size().
 */
int splat2d_preprocess(const splat2d_config* cfg, const splat2d_problem* prob, const splat2d_surfels* surfels,
                       void* ws, size_t ws_bytes, splat2d_stream stream);

/*
 * Follows: Eq. 1 (Sec. 3) blends surfels front to back in depth order, and
 * the paper renders the map "through standard rasterization" (Sec. 4.1,
 * the rendering loss): tile binning and a depth sort per tile.
 *
 * Tile binning and sort: every visible (view, surfel) pair emits one
 * instance per tile of its rect, key = (global tile) << 32 | FP32 depth bits,
 * value = surfel index, and the instances are put in key order, ties in
 * ascending surfel index (the order of a stable sort of the instances
 * emitted in surfel order).  The tile index is taken as the most significant
 * digit -- a counting pass gives each tile's [start, end) range and a
 * scatter fills per-tile buckets -- and each bucket is then sorted by its
 * depth bits with a radix sort in shared memory.  Follows splat2d_preprocess
 * on the same workspace.  If the instances exceed instance_capacity the
 * device status becomes SPLAT2D_ERR_CAPACITY with the needed count and
 * every later kernel of the iteration does nothing; re-run with a larger
 * capacity.
 */
int splat2d_bin_sort(const splat2d_config* cfg, const splat2d_problem* prob, void* ws, size_t ws_bytes,
                     splat2d_stream stream);

/*
 * Follows: Eq. 1 (Sec. 3), the alpha blending of colour, depth and
 * accumulation, I, D, A = sum_i (c_i, z_i, 1) w_i prod_{j<i} (1 - w_j).
 *
 * Forward compositing: one persistent launch over every (view, tile); each
 * tile stages chunks of its sorted surfels in shared memory and composites
 * front to back with warp-level early termination.  Writes rgb, depth,
 * normal, alpha (packed per view as described above; any may be NULL) and
 * keeps in `ws`, for the backward pass, per-pixel T_final and the last
 * blended index and a copy of every record it staged, in sorted-list order
 * (the workspace holds instance_capacity such 80-byte records).
 */
int splat2d_render_fwd(const splat2d_config* cfg, const splat2d_problem* prob, void* ws, size_t ws_bytes,
                       float* rgb, float* depth, float* normal, float* alpha, splat2d_stream stream);

/*
 * Follows: the analytic gradient of Eq. 1 (Sec. 3) with respect to the
 * surfel parameters and the camera pose, which the backend's rendering-based
 * refinement of the map over the latest keyframes needs (Sec. 4.3,
 * "Lightweight Map Refinement").
 *
 * Reverse pass: walks each pixel back to front from its last blended surfel,
 * recovering the transmittance by division instead of storing per-pixel
 * lists (32 (pixel, surfel) pairs per warp step, with segmented warp scans);
 * it reads the records from the sorted-order copy the forward left.
 * Per-surfel gradients are summed across the tile in shared memory (in
 * fixed point, each term rounded to a power-of-two fraction of the tile's
 * typical sum; terms outside that range are added exactly in global memory)
 * before one vector atomic per (tile, surfel); then a per-surfel pass chains
 * them to the parameters and reduces the per-view pose tangent.  d_* are
 * upstream gradients laid out like the forward outputs (NULL = zero).  Must
 * follow splat2d_render_fwd on the same workspace with unchanged surfels.
 */
int splat2d_render_bwd(const splat2d_config* cfg, const splat2d_problem* prob, const splat2d_surfels* surfels,
                       void* ws, size_t ws_bytes, const float* d_rgb, const float* d_depth,
                       const float* d_normal, const float* d_alpha, const splat2d_grads* grads,
                       splat2d_stream stream);

/*
 * The two halves of splat2d_render_bwd, for callers that time or overlap
 * them separately: the tile adjoint leaves per-(view, surfel) record
 * gradients in `ws`; the chain rule turns them into parameter and pose
 * gradients (accumulated into `grads`).  Calling both in this order is
 * exactly splat2d_render_bwd.
 */
int splat2d_render_bwd_tiles(const splat2d_config* cfg, const splat2d_problem* prob, void* ws, size_t ws_bytes,
                             const float* d_rgb, const float* d_depth, const float* d_normal, const float* d_alpha,
                             splat2d_stream stream);
int splat2d_preprocess_bwd(const splat2d_config* cfg, const splat2d_problem* prob, const splat2d_surfels* surfels,
                           void* ws, size_t ws_bytes, const splat2d_grads* grads, splat2d_stream stream);

/*
 * Follows: the 2D Gaussian surfel primitive the paper adopts (Sec. 3) comes
 * with a depth-distortion regulariser: per pixel, over the surfels it blends
 * in blending order,
 *     D_s = 2 sum_i sum_{j<i} w_i w_j (z_i - z_j),
 * z the depth each surfel contributes to the depth output (the center's z_i,
 * or with SPLAT2D_FLAG_DEPTH_RAY the ray-splat intersection depth).  With the
 * center depth -- the sort key, non-decreasing along the blending order --
 * this is sum_{i,j} w_i w_j |z_i - z_j|; with the ray depth it is the same
 * ordered sum (the intersection depths need not be sorted).
 *
 * splat2d_render_fwd_dist is splat2d_render_fwd that also writes D_s to
 * `dist` (device, one float per packed pixel, laid out like `alpha`; NULL
 * gives exactly splat2d_render_fwd).  splat2d_render_bwd_dist and
 * splat2d_render_bwd_tiles_dist are splat2d_render_bwd and
 * splat2d_render_bwd_tiles that also take d_dist, the upstream gradient of
 * D_s (same layout; NULL = zero), and add its gradient -- through the
 * weights and the depths -- to every parameter and pose gradient.  They
 * must follow a forward on the same workspace (either forward keeps what the
 * distortion's adjoint needs).  Errors as for the calls they extend.
 */
int splat2d_render_fwd_dist(const splat2d_config* cfg, const splat2d_problem* prob, void* ws, size_t ws_bytes,
                            float* rgb, float* depth, float* normal, float* alpha, float* dist,
                            splat2d_stream stream);
int splat2d_render_bwd_dist(const splat2d_config* cfg, const splat2d_problem* prob, const splat2d_surfels* surfels,
                            void* ws, size_t ws_bytes, const float* d_rgb, const float* d_depth,
                            const float* d_normal, const float* d_alpha, const float* d_dist,
                            const splat2d_grads* grads, splat2d_stream stream);
int splat2d_render_bwd_tiles_dist(const splat2d_config* cfg, const splat2d_problem* prob, void* ws,
                                  size_t ws_bytes, const float* d_rgb, const float* d_depth, const float* d_normal,
                                  const float* d_alpha, const float* d_dist, splat2d_stream stream);

/*
 * Map fusion, pruning input (Sec. 4.3, "Map Fusion": the global map is
 * rendered at the new keyframe's pose and primitives that contribute to
 * pixels with high RGB or depth error are removed).  For every (pixel,
 * surfel) pair the forward blended -- an entry of the pixel's tile list
 * before its last blended entry whose alpha there is at least alpha_min --
 * max_err[surfel] = max(max_err[surfel], err[pixel]).
 *   err      device, one float per packed pixel (laid out like the alpha
 *            output); values <= 0 and NaN count as zero.
 *   max_err  device, [n_surfels] floats, initialised by the caller (zeros,
 *            or the result of earlier calls) to values >= 0; only raised.
 * Must follow splat2d_render_fwd on the same workspace.  The caller prunes
 * the surfels whose max_err exceeds its threshold.  NULL pointers give
 * SPLAT2D_ERR_INVALID_ARG; after an instance-capacity overflow (device
 * status) the call does nothing.
 */
int splat2d_max_error(const splat2d_config* cfg, const splat2d_problem* prob, void* ws, size_t ws_bytes,
                      const float* err, float* max_err, splat2d_stream stream);

/*
 * Map fusion, insertion gate (Sec. 4.3, "Map Fusion": new primitives are
 * added only where the accumulation map rendered from the global map is
 * below a threshold tau_accum).
 *   alpha     device, n floats: the forward's alpha output at the new
 *             keyframe's pose, one per pixel (= per new per-pixel primitive).
 *   keep_idx  device, capacity n: receives the ascending indices i with
 *             alpha[i] < tau (NaN is never kept).
 *   n_keep    device int64: receives their number.
 *   tmp       device scratch of splat2d_accum_gate_tmp_size(n) bytes.
 * 0 <= n < 2^32.  Asynchronous on `stream`; no allocation.
 */
size_t splat2d_accum_gate_tmp_size(int64_t n);
int splat2d_accum_gate(const float* alpha, int64_t n, float tau, uint32_t* keep_idx, int64_t* n_keep, void* tmp,
                       size_t tmp_bytes, splat2d_stream stream);

/*
 * Adaptive voxelization of a keyframe's per-pixel map (Sec. 4.3, "Adaptive
 * Voxelization").  in: the keyframe's primitives, one per pixel, index
 * y * width + x (in->n must equal width * height), centers in the
 * keyframe's camera frame.  The map is cut into 2x2 blocks of primitives
 * (ragged blocks at odd edges); a block becomes one primitive with the mean
 * center, opacity, colour and tangent scales of its primitives and the
 * normalised sum of their quaternions, each first negated if its dot
 * product with the block's first quaternion is negative; a block whose
 * camera-frame depth range (max - min of mu.z) exceeds tau_d keeps its
 * primitives unchanged.  Writes, in order (blocks row-major; a kept block's
 * primitives row-major), the primitives to out (device arrays with capacity
 * width * height), their block index to out_block (device int32, may be
 * NULL), and their number to *n_out (device int64).  tmp: device scratch of
 * splat2d_voxelize_tmp_size(width, height) bytes.  No allocation, async.
 */
size_t splat2d_voxelize_tmp_size(int32_t width, int32_t height);
int splat2d_voxelize(const splat2d_surfels* in, int32_t width, int32_t height, float tau_d,
                     const splat2d_surfel_buffers* out, int32_t* out_block, int64_t* n_out, void* tmp,
                     size_t tmp_bytes, splat2d_stream stream);

/*
 * Sim(3) transform of primitives, in place (Sec. 4.3: "Map Fusion" moves a
 * keyframe's primitives from its camera frame to the world with the
 * keyframe's Sim(3) pose, mu' = s R mu + t and r' = q r; "Loop Correction of
 * Gaussian Map" applies to each keyframe's primitives the change of its
 * pose, Delta T = T_new T_old^-1).  sim3: device, [K, 8] rows (qw, qx, qy,
 * qz, tx, ty, tz, s), q any nonzero norm (normalised inside).  index:
 * device int32 [n] choosing each primitive's row (the keyframe it is bound
 * to), or NULL for row 0.  means, quats, scales: device arrays of n
 * primitives, updated in place (any may be NULL to leave it); quats become
 * q r (Hamilton product, not renormalised); scales are multiplied by s.
 */
int splat2d_sim3_apply(int64_t n, float* means, float* quats, float* scales, const float* sim3,
                       const int32_t* index, splat2d_stream stream);

/* Number of kernels this library has enqueued since it was loaded (host-side
 * count, including launches recorded into a CUDA graph). */
uint64_t splat2d_launch_count(void);

/* Synchronise `stream`, read the device status and counters of the last
 * iteration into *out.  Returns out->status (or a host error). */
int splat2d_stats(const void* ws, splat2d_stats_t* out, splat2d_stream stream);

/* Like splat2d_stats but returns only the status and, if needed_capacity is
 * not NULL, the instance count the last binning needed. */
int splat2d_status(const void* ws, int64_t* needed_capacity, splat2d_stream stream);

/* Byte offsets of the workspace sub-buffers (for inspection and tests). */
typedef struct {
  size_t records;     /* [R] 80-byte render records, R = sum of view ranges */
  size_t ntiles;      /* [R] uint32 tile count per record (0 = culled) */
  size_t keys;        /* [capacity] uint64 sorted keys (after splat2d_bin_sort) */
  size_t vals;        /* [capacity] uint32 sorted surfel indices */
  size_t ranges;      /* [T] uint32 x2 per global tile: [start, end) */
  size_t tfinal;      /* [P] float per pixel */
  size_t last;        /* [P] uint32 per pixel: one past the last blended entry of its tile list */
  size_t total;       /* = splat2d_workspace_size */
  int64_t n_records;  /* R */
  int64_t n_tiles;    /* T */
  int64_t n_pixels;   /* P */
} splat2d_layout;
int splat2d_workspace_layout(const splat2d_config* cfg, const splat2d_problem* prob, splat2d_layout* out);

/*
 * The radix sort on its own: stably sorts n (key, value) pairs in place by
 * the low `key_bits` bits of the keys (1..64; higher bits must be zero).
 * keys/vals are device arrays; tmp is a device buffer of
 * splat2d_sort_tmp_size(n) bytes.  Asynchronous on `stream`.
 */
size_t splat2d_sort_tmp_size(int64_t n);
int splat2d_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int key_bits, void* tmp, size_t tmp_bytes,
                       splat2d_stream stream);

/*
 * splat2d_sort_pairs without any allocation: the same stable sort, with its
 * scratch in a fixed device array inside the library instead of a caller
 * buffer.  The paper has no counterpart; this serves callers that cannot
 * allocate device memory (code running during CUDA-graph capture, real-time
 * loops with a no-allocation rule, plug-ins whose host application owns all
 * device memory).  n must not exceed SPLAT2D_SORT_NOALLOC_MAX_PAIRS
 * (SPLAT2D_ERR_INVALID_ARG otherwise).  The array (about 13 MB) is held on
 * every GPU that loads the library until the process exits.  All calls share
 * it, so calls that overlap on the GPU race; calls on one stream are safe.
 * The first call on a device looks up the array's address with that device
 * current: make it before any stream capture.
 */
#define SPLAT2D_SORT_NOALLOC_MAX_PAIRS (1 << 20)
int splat2d_sort_pairs_noalloc(uint64_t* keys, uint32_t* vals, int64_t n, int key_bits, splat2d_stream stream);

/* Human-readable name of a status code. */
const char* splat2d_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* SPLAT2D_H */
