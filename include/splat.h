/*
 * splat.h -- C ABI of the GB300 (sm_103a) differentiable tile-based RGB-D
 * Gaussian rasterizer: the data-parallel hot path of MAC-Ego3D
 * (arXiv 2412.09723).
 *
 * Conventions shared by every call
 * --------------------------------
 * Memory:   the caller owns all memory.  Every array pointer is a DEVICE
 *           pointer (cudaMalloc / torch CUDA tensor, float32 or int32,
 *           C-contiguous) unless the comment says "host".  Structs describing
 *           arrays are passed by host pointer.  The library never allocates;
 *           calls that need scratch space take a workspace pointer whose size
 *           the matching *_workspace_size() query returns (256-byte aligned).
 * Streams:  every call is asynchronous and ordered on `stream` (NULL = the
 *           legacy default stream).  No call synchronises with the host, so
 *           every call can be captured into a CUDA graph.  Counts that depend
 *           on the data (duplicates K, association pairs M) are written to
 *           device int64 slots; reading them is an explicit caller action.
 * Errors:   each call returns SPLAT_OK or an error code for argument errors
 *           (SPLAT_EINVAL) and launch errors (SPLAT_ECUDA); the text of the
 *           last error on the calling thread is splat_last_error().  Errors
 *           only the device can detect (a capacity overflow) are written to
 *           the caller's device `status` word (int32, 0 = ok) and must be
 *           checked after synchronising.  Entry points never write outside the
 *           buffers their sizes describe, even on overflow.
 * Geometry: world-to-camera pose `w2c` is a device float[16], row-major 4x4
 *           [R t; 0 1]; camera space is x right, y down, z forward.  Pixel
 *           (x, y) has its centre at (x + 0.5, y + 0.5).  Tiles are 16x16
 *           pixels, tile id = ty * ceil(W/16) + tx.
 *
 * Paper anchors: map representation and the rendering equation, Sec. 3.3;
 * depth rendering for the geometric loss, Sec. 3.5 (Optimization, Eq. optim);
 * map optimisation by differentiable rendering, Sec. 3.4 step 4; inter-agent
 * association and alignment, Sec. 3.5 steps 2-3; batched differentiable
 * rendering across agents, Sec. 3.6.  The paper fixes no rasterizer constant;
 * this library uses: alpha = min(0.99, opacity * exp(power)), skip alpha <
 * 1/255, stop before a Gaussian that would take transmittance below 1e-4,
 * +0.3 px^2 low-pass on the 2D covariance, EWA Jacobian with x/z, y/z clamped
 * to 1.3 tan(fov/2), near plane z_near (culls z <= z_near), radius
 * ceil(3 sqrt(lambda_max)).
 */
#ifndef SPLAT_H
#define SPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *splat_stream_t;

enum {
  SPLAT_OK = 0,
  SPLAT_EINVAL = 1,    /* null pointer, bad size or misaligned buffer */
  SPLAT_ECAPACITY = 2, /* (device status) an output buffer was too small */
  SPLAT_ECUDA = 3,     /* a kernel launch or CUDA runtime call failed */
  SPLAT_ETIMEOUT = 4,  /* (device status) a bounded wait inside a launch gave up (splat_render_fwd_bwd) */
  SPLAT_ENUMERIC = 8   /* (device status) a linear system was not positive definite */
};

/* Pinhole camera.  tan(fov_x / 2) = width / (2 fx).  max_dist > 0 limits the
 * candidates to Gaussians within that distance of the camera centre (the
 * distance part of the candidate selection of Sec. 3.4 step 1); 0 = no limit. */
typedef struct {
  int32_t width, height;
  float fx, fy, cx, cy;
  float z_near;
  float max_dist;
} splat_camera;

/* Gaussian map, structure of arrays (Sec. 3.3: mean x, covariance from
 * scale s and rotation, opacity lambda, colour c).  quat is (w, x, y, z) and
 * need not be normalised; scale = exp(log_scale); opacity =
 * sigmoid(opacity_logit).  quat must be 16-byte aligned. */
typedef struct {
  const float *mean;          /* [n,3] world */
  const float *log_scale;     /* [n,3] */
  const float *quat;          /* [n,4] */
  const float *opacity_logit; /* [n]   */
  const float *rgb;           /* [n,3] */
  int64_t n;
} splat_gaussians;

/* Gradients with the same shapes as splat_gaussians (accumulated, +=). */
typedef struct {
  float *mean, *log_scale, *quat, *opacity_logit, *rgb;
} splat_gaussians_grad;

/* Per-Gaussian projection (all rows of a culled Gaussian are zero).
 * xyzo and conic and rect must be 16-byte aligned. */
typedef struct {
  float *xyzo;            /* [n,4] u, v (pixels), depth z, opacity        */
  float *conic;           /* [n,4] inverse 2D covariance a, b, c, and the
                             smallest exponent at which this Gaussian's
                             alpha can still reach 1/255 (minus a margin)  */
  int32_t *radius;        /* [n] ceil(3 sqrt(lambda_max)); 0 = culled      */
  int32_t *rect;          /* [n,4] tile xmin, ymin, xmax, ymax (half open) */
  int32_t *tiles_touched; /* [n] (xmax - xmin) * (ymax - ymin): rect area, an upper bound of the member tiles */
} splat_projected;

/* Per-pixel render outputs, row-major [H,W] (rgb [H,W,3]). */
typedef struct {
  float *rgb;
  float *depth;      /* sum z_i alpha_i T_i (not normalised)            */
  float *sil;        /* sum alpha_i T_i                                 */
  float *t_final;    /* transmittance after the last contributor         */
  int32_t *n_contrib;/* position in the tile list of the last
                        contributor, plus one (0 = none)                */
  int32_t *max_id;   /* Gaussian with the largest alpha_i T_i; -1 = none;
                        ties keep the front-most                         */
  int32_t *n_used;   /* optional (may be NULL): number of Gaussians that
                        contributed to the pixel                         */
} splat_image;

/* Version of this ABI (incremented on any incompatible change). */
int32_t splat_abi_version(void);

/* Text of the last error returned on the calling thread ("" if none). */
const char *splat_last_error(void);

/* Number of CUDA kernels this library has launched in this process (host-side
 * count of launch calls; kernels replayed from a captured graph are not
 * counted again). */
uint64_t splat_kernel_launches(void);

/* Per-kernel timing (tracing aid; the paper reports per-frame timings only,
 * Sec. 4.4).  While enabled, every kernel launch of this library is bracketed
 * by a CUDA event pair recorded on its launching stream.  Do not enable it
 * while a stream is being captured into a graph.  Returns SPLAT_OK. */
int splat_profile_enable(int on);

/* Restricts the timing to launches of the kernel named `kernel` (host string,
 * copied; NULL or "" = every kernel).  Timing a single kernel keeps the host
 * cost of the event records small enough not to leave the GPU waiting between
 * launches.  Returns SPLAT_OK. */
int splat_profile_select(const char *kernel);

/* Waits for the recorded events, then returns, per kernel name, the number of
 * timed launches and their summed duration in milliseconds, and forgets the
 * records.  names (host, names_bytes) receives the kernel names separated by
 * '\n' (truncated to fit); launches (host int64[max_kernels]) and ms (host
 * double[max_kernels]) the figures in the same order; *n_kernels (host) the
 * number of distinct kernels (which may exceed max_kernels).
 * Errors: SPLAT_EINVAL, SPLAT_ECUDA (an event could not be read). */
int splat_profile_read(char *names, size_t names_bytes, int64_t *launches, double *ms,
                       int32_t max_kernels, int32_t *n_kernels);

/*
 * splat_project -- per-Gaussian activation and EWA projection (Sec. 3.3, the
 * f_i^proj of the rendering equation; the frustum and distance candidate
 * selection of Sec. 3.4 step 1).
 *   s = exp(log_scale), R = R(q/|q|) (identity if |q| = 0),
 *   Sigma = R diag(s^2) R^T, opacity = sigmoid(logit), p = W x + t;
 *   culled if p_z <= z_near, or if max_dist > 0 and
 *   (p_x p_x + p_y p_y) + p_z p_z > max_dist max_dist (float32, in this order);
 *   Sigma2 = J W Sigma W^T J^T + 0.3 I;
 *   culled if det(Sigma2) <= 0; conic = Sigma2^-1; (u, v) = (fx p_x/p_z + cx,
 *   fy p_y/p_z + cy); radius r = ceil(3 sqrt(lambda_max(Sigma2)));
 *   rect = [floor((u-r)/16), floor((u+r)/16)+1) x (same in v), clamped to
 *   the tile grid; culled if the rect is empty.
 * g: device arrays; cam: host; w2c: device float[16]; out: device arrays of
 * g->n rows.  Errors: SPLAT_EINVAL (null or misaligned pointer, n < 0,
 * non-positive image size), SPLAT_ECUDA.
 */
int splat_project(const splat_gaussians *g, const splat_camera *cam, const float *w2c,
                  const splat_projected *out, splat_stream_t stream);

/*
 * Tile schedule: the order in which the renders take a view's tiles, heaviest
 * first, so that a persistent launch ends on light tiles.  The cost of a
 * tile is the number of list positions its pixels walk (not the list length:
 * a pixel stops at its last contributor), which the forward render knows at
 * its end.  Layout: uint32[1 + 2 n_tiles]:
 *   [0]                      n_tiles once an order has been written, else 0;
 *   [1, 1 + n_tiles)         tile ids, heaviest first;
 *   [1 + n_tiles, 1 + 2 n_tiles)  per-tile cost: the summed contributor counts
 *                            of the tile's pixels in the last forward render.
 * The forward render (splat_render_fwd_l1, splat_render_fwd_bwd, a batch
 * forward) writes the costs; splat_bin_sort rebuilds the order from them
 * (tiles by cost bucket 1 + floor(8 log2 cost), heaviest bucket first; cost 0
 * last).  A step's order therefore comes from the previous step's costs, which
 * barely change between the iterations on one frame.  A zero-filled buffer
 * holds no order (the natural order is taken).  The schedule changes only the
 * order of the work: results are the same with or without it.
 */
size_t splat_tile_schedule_size(int32_t n_tiles); /* bytes */

/*
 * splat_tile_schedule_order -- rebuild a schedule's order from its costs (the
 * part of splat_bin_sort that does it, alone: one CTA), so that a caller can
 * build it beside the projection and binning, on another stream, and call
 * splat_bin_sort with schedule = NULL.  Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
int splat_tile_schedule_order(uint32_t *schedule, int32_t n_tiles, splat_stream_t stream);

/*
 * splat_bin_sort -- duplicate every visible Gaussian into each of its member
 * tiles and sort the (tile, depth) keys (the tile binning and front-to-back
 * order the rendering equation of Sec. 3.3 composites in).
 * Members: the tiles of the rect whose 16 x 16 rectangle of pixel centres can
 * reach opacity * exp(-Q/2) >= 0.99/255 (Q = a dx^2 + 2 b dx dy + c dy^2 with
 * the conic; minimum of Q over the rectangle: 0 with the centre inside, else
 * the closed-form minimum over each edge, each operation rounded in the
 * order written: xa = ((16 tx) + 0.5) - u, xb = xa + 15, same in y; on the
 * edge y = dy, dx = min(xb, max(xa, -((b / a) dy))) and
 * Q = ((a dx) + ((2 b) dy)) dx + (c dy) dy; on the edge x = dx,
 * dy = min(yb, max(ya, -((b / c) dx))) and Q = (a dx) dx + (((2 b) dx) + (c dy)) dy;
 * the test is opacity * exp(-0.5 Q_min) >= 0.99f / 255 with splat_exp_f32's
 * exponential); in each rect row the members run from the first to the last
 * tile that passes.  No pixel can take a Gaussian in a tile left out, so the
 * images are those of whole rects.
 * Result: for every tile t, vals[ranges[2t] .. ranges[2t+1]) are the ids of
 * the Gaussians holding t, in ascending (depth, id) order; tiles follow each
 * other in tile-id order; an empty tile has range (0, 0).
 * keys (optional, may be NULL) receives (uint64)tile << 32 | bits(depth).
 *   proj:     output of splat_project for n Gaussians (device; xyzo, conic,
 *             rect and tiles_touched are read)
 *   cam:      host; only width/height are used
 *   keys:     device uint64[capacity] or NULL
 *   vals:     device uint32[capacity]
 *   capacity: number of slots in keys/vals (< 2^31)
 *   k_dev:    device int64[1]: receives K, the number of duplicates
 *   ranges:   device uint32[2 * n_tiles]
 *   schedule: a tile schedule (above) or NULL: its order is rebuilt here from
 *             the costs the last forward render wrote
 *   status:   device int32[1]: set to SPLAT_ECAPACITY when K > capacity (the
 *             sorted lists are then incomplete; resize and call again);
 *             never cleared by the library
 *   ws:       device workspace of splat_bin_sort_workspace_size() bytes
 * Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
size_t splat_bin_sort_workspace_size(int64_t n, int64_t capacity, int32_t n_tiles);
int splat_bin_sort(const splat_projected *proj, int64_t n, const splat_camera *cam,
                   uint64_t *keys, uint32_t *vals, int64_t capacity, int64_t *k_dev,
                   uint32_t *ranges, uint32_t *schedule, int32_t *status, void *ws,
                   size_t ws_bytes, splat_stream_t stream);

/*
 * splat_bin_sort_static -- splat_bin_sort without a caller workspace.  (The
 * paper has no counterpart: this is a convenience of this library.)
 * For callers that cannot allocate device memory when they render -- a
 * real-time loop that reserved its memory once at start-up and must not enter
 * an allocator afterwards, or a host framework that owns the allocator and
 * cannot lend scratch space to the code issuing the render.  The scratch comes
 * from one device array of splat_bin_sort_static_scratch_bytes() bytes
 * (64 MiB) that is part of this library's module: every GPU that loads the
 * library holds it until the process exits.  The call allocates nothing.
 *   Arguments, results and errors as splat_bin_sort (minus ws / ws_bytes).
 *   Sizes whose scratch need exceeds the array (16 bytes per duplicate slot
 *   and 8 per Gaussian: about 27 MiB for 300k Gaussians with 1.6M slots) are
 *   rejected with SPLAT_EINVAL and a message.
 *   The first call on a device looks up the array's device address (with
 *   that device current): make that first call before any stream capture.
 *   Later calls look the address up again unless their stream is capturing,
 *   so that a device reset (which reloads the module) is followed.
 *   All calls share the one array and leave their data in it; calls that
 *   may overlap on the GPU (several streams or threads) race and must be
 *   serialised by the caller.
 */
size_t splat_bin_sort_static_scratch_bytes(void);
int splat_bin_sort_static(const splat_projected *proj, int64_t n, const splat_camera *cam,
                          uint64_t *keys, uint32_t *vals, int64_t capacity, int64_t *k_dev,
                          uint32_t *ranges, int32_t *status, splat_stream_t stream);

/*
 * splat_render_fwd -- per-pixel front-to-back alpha compositing of colour,
 * depth and silhouette over the pixel's tile list (rendering equation of
 * Sec. 3.3; rendered depth of Sec. 3.5), recording the final transmittance
 * and the maximum-weight Gaussian used for association (Sec. 3.5 step 2).
 *   C = sum c_i w_i + T_final bg, D = sum z_i w_i, S = sum w_i,
 *   w_i = alpha_i T_i, T_{i+1} = T_i (1 - alpha_i).
 *   proj/vals/ranges: outputs of splat_project and splat_bin_sort;
 *   rgb: device [n,3] Gaussian colours; bg: HOST float[3] background;
 *   out: device image arrays of cam->height x cam->width pixels.
 * Deterministic (no atomics).  Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
int splat_render_fwd(const splat_projected *proj, const float *rgb, int64_t n,
                     const uint32_t *vals, const uint32_t *ranges, const splat_camera *cam,
                     const float *bg, const splat_image *out, splat_stream_t stream);

/*
 * splat_render_bwd -- adjoint of splat_project + splat_render_fwd for
 * per-pixel upstream gradients (map optimisation by differentiable rendering,
 * Sec. 3.4 step 4; gradients through renders for alignment and joint
 * optimisation, Sec. 3.5 steps 3-4).
 *   proj: the splat_project output for this map, camera and pose (its radius
 *     is read: Gaussians it culled get no gradient and are skipped).
 *   schedule: the view's tile schedule (its order is used), or NULL for the
 *     natural order (the result is the same either way).
 *   d_rgb [H,W,3], d_depth [H,W], d_sil [H,W] (d_depth, d_sil may be NULL).
 *   fwd: the image of the forward call (t_final, n_contrib are read).
 *   out: Gaussian-parameter gradients, ACCUMULATED (+=); the caller zeroes.
 *   d_pose: device float[6] or NULL, ACCUMULATED: gradient w.r.t. (rho, phi)
 *     of the left perturbation w2c <- exp(delta^) w2c.
 *   d2d: device float[n,10] or NULL: receives the screen-space gradients
 *     (du, dv, d conic a, b, c, d opacity, d rgb[3], d depth) (overwritten).
 *   ws: workspace of splat_render_bwd_workspace_size(n) bytes, 16-byte
 *     aligned (always required: the screen-space gradients accumulate there,
 *     [n,12] float rows as splat_project_bwd reads them).
 *   out, d_pose and d2d all NULL: only the screen-space adjoint runs, and its
 *     gradients are left in ws for splat_project_bwd or splat_project_bwd_adam.
 * The tile lists are walked in two independent parts per tile (positions
 * before and after a split point, front to back and back to front) by one
 * persistent launch; atomics make the summation order, and so the last bits,
 * vary between runs.
 * Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
size_t splat_render_bwd_workspace_size(int64_t n);
int splat_render_bwd(const splat_gaussians *g, const splat_projected *proj,
                     const splat_camera *cam, const float *w2c, const uint32_t *vals,
                     const uint32_t *ranges, const uint32_t *schedule,
                     const splat_image *fwd, const float *bg,
                     const float *d_rgb, const float *d_depth, const float *d_sil,
                     const splat_gaussians_grad *out, float *d_pose, float *d2d, void *ws,
                     size_t ws_bytes, splat_stream_t stream);

/*
 * splat_project_bwd -- the projection adjoint alone (the second half of
 * splat_render_bwd): chains screen-space gradients grad2d (device float
 * [n,12], 16-byte aligned rows: du, dv, d conic a, b, c, d opacity,
 * d rgb[3], d depth, 2 unused) to the Gaussian parameters (accumulated into
 * `out`, or not formed when `out` is NULL) and, if d_pose is not NULL, to the
 * pose 6-vector (accumulated); out, d_pose and d2d may not all be NULL.
 * d2d (optional) receives the [n,10] screen-space gradients.  proj must be
 * the splat_project output for the same map, camera and pose (Gaussians with
 * radius 0 are skipped).  Used after splat_render_bwd_batch.
 * Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
int splat_project_bwd(const splat_gaussians *g, const splat_projected *proj, const splat_camera *cam,
                      const float *w2c, const float *grad2d, const splat_gaussians_grad *out,
                      float *d_pose, float *d2d, splat_stream_t stream);

/*
 * splat_project_bwd_adam -- splat_project_bwd with the map's Adam step taken
 * in the same launch (map optimisation, Sec. 3.4 step 4, the SplaTAM-style
 * optimiser): every Gaussian's 14 parameters move by one bias-corrected Adam
 * step with the gradient the projection adjoint gives it -- the gradient
 * splat_project_bwd would accumulate into zeroed arrays, 0 for a Gaussian the
 * projection culled -- the same update as splat_adam_groups with those
 * gradients, bit for bit.  No gradient array is read or written.  The kept
 * Gaussians (radius > 0) run the adjoint and their update; with culled != 0
 * the culled ones take their zero-gradient update in other CTAs of the same
 * launch, else the caller runs splat_adam_culled for them (which needs only
 * the projection, so it can run beside the render on another stream).
 * Elements of culled Gaussians whose moments are both +0 are left exactly as
 * they are (their update is nothing).  The pose gradient is accumulated into
 * d_pose (if not NULL) as by splat_project_bwd.
 *   g: the map; its arrays are UPDATED IN PLACE (the const of splat_gaussians
 *     does not hold for this call).  m, v: device moments of the same shapes.
 *   lr: HOST float[5], the step sizes of mean, log_scale, quat,
 *     opacity_logit, rgb; step: DEVICE int32[1] holding t >= 1.
 *   seen: device uint32[ceil(n / 32)] or NULL: bit i set when Gaussian i's
 *     moments may be nonzero; a clear bit PROMISES m = v = 0 for all its
 *     elements (the caller keeps that true: zeros with zeroed moments, all
 *     ones when unsure).  The call sets the bits of the kept Gaussians, and
 *     the culled part then touches only culled Gaussians whose bit is set, so
 *     a map mostly never optimised costs one bit per Gaussian there (the
 *     SplaTAM-style optimiser restarts its moments per frame).
 *   proj, cam, w2c, grad2d: as splat_project_bwd.
 *   pose: NULL, or the pose's Adam step and retraction (as splat_pose_step
 *     with d_pose as the gradient) taken in the same launch by the last CTA
 *     that adds to d_pose, after every CTA has read w2c and added its
 *     gradient; d_pose must then be zero on entry (it receives the whole
 *     gradient).
 * Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
typedef struct {
  float *w2c;          /* device float[16] updated in place (may be the w2c argument's buffer) */
  float *m, *v;        /* device float[6]: the pose's moments */
  const int32_t *step; /* device int32[1] holding t >= 1 */
  float lr_t, lr_r, beta1, beta2, eps;
  uint32_t *counter;   /* device uint32[1]: 0 on entry, left 0 */
} splat_pose_adam;

int splat_project_bwd_adam(const splat_gaussians *g, const splat_projected *proj,
                           const splat_camera *cam, const float *w2c, const float *grad2d,
                           const splat_gaussians_grad *m, const splat_gaussians_grad *v,
                           const float *lr, float beta1, float beta2, float eps,
                           const int32_t *step, uint32_t *seen, int32_t culled, float *d_pose,
                           const splat_pose_adam *pose, splat_stream_t stream);

/*
 * splat_adam_culled -- the zero-gradient Adam step of the Gaussians a
 * projection culled (radius == 0), the other part of splat_project_bwd_adam
 * called with culled = 0; arguments (seen included) as there, radius from
 * splat_project.
 * Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
int splat_adam_culled(const splat_gaussians *g, const int32_t *radius, const splat_gaussians_grad *m,
                      const splat_gaussians_grad *v, const float *lr, float beta1, float beta2,
                      float eps, const int32_t *step, uint32_t *seen, splat_stream_t stream);

/*
 * splat_render_fwd_l1 -- splat_render_fwd with the L1 terms of the loss of
 * Eq. (optim) (Sec. 3.5) taken in the same pass, while each pixel's colour and
 * depth are still in registers: for the rendered C, D and targets C*, D*,
 *   loss    += w_rgb mean|C - C*| + w_depth mean|D - D*|
 *              (means over the 3 H W colour and H W depth values),
 *   d_rgb    = (w_rgb / 3HW) sign(C - C*),  d_depth = (w_depth / HW) sign(D - D*),
 *   sign(0) = 0.  The gradients are written (not accumulated) and equal those of
 *   splat_loss_l1 on the rendered images bit for bit; the loss is summed in a
 *   different order (per tile, then one float atomic per tile).
 *   l1: descriptor below (device arrays [H,W,3] / [H,W]; loss: device float,
 *   accumulated, the caller zeroes it), or NULL for a render without loss
 *   terms that fills the schedule.
 *   schedule: a tile schedule or NULL: the tiles are taken in its order and
 *     their costs written to it.
 * Errors: as splat_render_fwd.
 */
typedef struct {
  const float *t_rgb;    /* target colour [H,W,3] */
  const float *t_depth;  /* target depth [H,W] */
  float w_rgb, w_depth;  /* weights of the two L1 terms */
  float *d_rgb;          /* out: dL/dC [H,W,3] */
  float *d_depth;        /* out: dL/dD [H,W] */
  float *loss;           /* in/out: device float, += L (may be NULL) */
} splat_l1;

int splat_render_fwd_l1(const splat_projected *proj, const float *rgb, int64_t n,
                        const uint32_t *vals, const uint32_t *ranges, const splat_camera *cam,
                        const float *bg, const splat_image *out, const splat_l1 *l1,
                        uint32_t *schedule, splat_stream_t stream);

/*
 * splat_render_fwd_bwd -- splat_render_fwd_l1 followed by the screen-space
 * adjoint of splat_render_bwd for the L1 gradients it writes, in ONE launch
 * (the rendering equation of Sec. 3.3 and its adjoint for the map and pose
 * optimisation of Sec. 3.4 step 4 and Sec. 3.5).  The backward of a tile
 * needs only that tile's forward outputs and loss gradients, so a tile's
 * backward starts as soon as its forward has finished, while other tiles are
 * still rendered: the forward's tail and the second launch's ramp disappear.
 * The forwards are taken in the schedule's order; the two backward parts of
 * the tiles follow in the order their forwards finished (a completion queue
 * in the workspace: a backward item waits, with a bounded number of polls,
 * for the next finished tile, never for a particular one).
 *   Arguments as splat_render_fwd_l1 (l1 required: its d_rgb / d_depth are
 *   the backward's upstream gradients, silhouette gradient 0), then
 *   status: device int32[1]; SPLAT_ETIMEOUT is raised if a wait gave up (the
 *     results are then incomplete; no input of this library's own making
 *     causes it);
 *   ws: workspace of splat_render_fwd_bwd_workspace_size(n, n_tiles) bytes,
 *     16-byte aligned; on return its first bytes hold the screen-space
 *     gradients exactly as splat_render_bwd leaves them in screen-only mode
 *     ([n,12] float rows), for splat_project_bwd or splat_project_bwd_adam.
 * Images and loss gradients are bit for bit those of splat_render_fwd_l1;
 * the screen-space gradients are the same sums as splat_render_bwd's (the
 * atomics' order, and so the last bits, vary).  The launch is cooperative.
 * Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
size_t splat_render_fwd_bwd_workspace_size(int64_t n, int32_t n_tiles);
int splat_render_fwd_bwd(const splat_projected *proj, const float *rgb, int64_t n,
                         const uint32_t *vals, const uint32_t *ranges, const splat_camera *cam,
                         const float *bg, const splat_image *out, const splat_l1 *l1,
                         uint32_t *schedule, int32_t *status, void *ws, size_t ws_bytes,
                         splat_stream_t stream);

/*
 * Several views in one launch (batched differentiable rendering across
 * agents, Sec. 3.6).  A view bundles one agent's projected map and sorted
 * lists with its camera and image; views may have different Gaussian counts
 * and image sizes.  The forward (backward) renders every tile of every view in
 * ONE persistent launch: (CTAs per SM) x (SMs) CTAs take (view, tile) items
 * from an atomic ticket counter; no CTA waits on another.  Results equal the
 * single-view calls (the forward bit for bit).
 */
#define SPLAT_MAX_VIEWS 16

typedef struct {
  splat_projected proj;  /* output of splat_project (device) */
  const float *rgb;      /* [n,3] Gaussian colours (device) */
  int64_t n;
  const uint32_t *vals;  /* sorted ids and tile ranges of splat_bin_sort */
  const uint32_t *ranges;
  splat_camera cam;
  float bg[3];           /* background colour */
  splat_image image;     /* forward outputs; t_final, n_contrib read back by the backward */
  const float *d_rgb;    /* backward only: upstream per-pixel gradients (d_depth, d_sil may be NULL) */
  const float *d_depth;
  const float *d_sil;
  float *grad2d;         /* backward only: [n,12] screen-space gradients, 16-byte aligned;
                            zeroed and filled by splat_render_bwd_batch */
  const splat_l1 *l1;    /* forward only, optional: the view's L1 loss terms taken in the
                            forward's epilogue (as splat_render_fwd_l1); NULL = none */
  uint32_t *schedule;    /* optional tile schedule of the view (splat_render_fwd_l1): the
                            forward fills it, the backward takes the tiles in its order */
} splat_view;

/* Execution shape (does not change any result): shared-memory batch of
 * Gaussians staged per round (64, 128 or 256) and resident CTAs per SM of the
 * persistent grids. */
typedef struct {
  int32_t fwd_batch, fwd_ctas_per_sm;  /* fwd_ctas_per_sm in 1..8  */
  int32_t bwd_batch, bwd_ctas_per_sm;  /* bwd_ctas_per_sm in 1..16 */
} splat_batch_shape;

/* Workspace (device, bytes) of the batched calls: the ticket counters. */
size_t splat_batch_workspace_size(void);

/* Host array `views` of n_views (1..SPLAT_MAX_VIEWS) views; shape may be NULL
 * (default shape).  Errors: SPLAT_EINVAL, SPLAT_ECUDA. */
int splat_render_fwd_batch(const splat_view *views, int32_t n_views, const splat_batch_shape *shape,
                           void *ws, size_t ws_bytes, splat_stream_t stream);
int splat_render_bwd_batch(const splat_view *views, int32_t n_views, const splat_batch_shape *shape,
                           void *ws, size_t ws_bytes, splat_stream_t stream);

/*
 * splat_loss_l1 -- the L1 colour and depth terms of Eq. (optim) (Sec. 3.5):
 *   L = w_rgb mean|C - C*| + w_depth mean|D - D*|, sign(0) = 0.
 * Writes dL/dC [npix,3] and dL/dD [npix] (overwritten) and ADDS L to
 * loss[0] (device float).  Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
int splat_loss_l1(const float *rgb, const float *depth, const float *target_rgb,
                  const float *target_depth, int64_t npix, float w_rgb, float w_depth,
                  float *d_rgb, float *d_depth, float *loss, splat_stream_t stream);

/*
 * splat_adam -- one bias-corrected Adam step on n resident float32
 * parameters (map optimisation, Sec. 3.4 step 4, following SplaTAM):
 *   m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 *   p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
 * step: DEVICE int32[1] holding t >= 1 (read on the device, so that a
 * captured graph can be replayed with an advancing count).
 * Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
int splat_adam(float *param, const float *grad, float *m, float *v, int64_t n, const int32_t *step,
               float lr, float beta1, float beta2, float eps, splat_stream_t stream);

/*
 * splat_adam_groups -- splat_adam over up to 8 parameter groups in one launch
 * (e.g. mean, log_scale, quat, opacity_logit, rgb of a map), each with its
 * own learning rate, sharing one device step count.  params[g], grads[g],
 * m[g], v[g] are device arrays of sizes[g] floats (host arrays of pointers);
 * lr: host float[n_groups].  With zero_grad != 0 every gradient element is set
 * to 0 after it is consumed, so the next backward can accumulate into it.
 * Aligned runs of 4 elements whose gradient and both moments are all +0.0
 * (bit pattern 0) are skipped: their update is exactly nothing (m and v stay
 * +0, p - 0 = p), so the result is bit for bit that of the full update while
 * the parameters of Gaussians unseen since their moments were zero are
 * neither read nor written.
 * Errors: SPLAT_EINVAL (n_groups not in 1..8, null pointer), SPLAT_ECUDA.
 */
int splat_adam_groups(int32_t n_groups, float *const *params, float *const *grads, float *const *m,
                      float *const *v, const int64_t *sizes, const float *lr, const int32_t *step,
                      float beta1, float beta2, float eps, int32_t zero_grad, splat_stream_t stream);

/*
 * splat_pose_step -- Adam on the 6-vector pose gradient followed by the
 * retraction w2c <- exp(delta^) w2c (render-driven tracking / alignment).
 *   w2c: device float[16] updated in place; d_pose: device float[6];
 *   m, v: device float[6] moments; step: DEVICE int32[1] holding t >= 1;
 *   lr_t, lr_r: step sizes for rho and phi.
 * Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
int splat_pose_step(float *w2c, const float *d_pose, float *m, float *v, const int32_t *step,
                    float lr_t, float lr_r, float beta1, float beta2, float eps,
                    splat_stream_t stream);

/*
 * splat_pose_compose -- out[k] = a[k] b for n row-major 4x4 poses (device
 * float[n,16], float[16], float[n,16]): the cameras through which a map
 * aligned by a relative transform is seen, w2c_eff = w2c_A T_rel (inter-agent
 * alignment, Sec. 3.5 step 3).  Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
int splat_pose_compose(int32_t n, const float *a, const float *b, float *out, splat_stream_t stream);

/*
 * splat_pose_rel_grad -- gradient with respect to the left perturbation of a
 * relative transform T_rel when view k is rendered with w2c[k] T_rel and
 * d_cam[k] is that view's camera-pose gradient (both 6-vectors (rho, phi)):
 * w2c exp(d^) T_rel = exp((Ad_w2c d)^) w2c T_rel, so
 * d_rel = sum_k Ad(w2c[k])^T d_cam[k], i.e. rho: R^T g_rho, phi: R^T (g_phi - t x g_rho).
 * w2c: device float[n,16]; d_cam: device float[n,6]; d_rel: device float[6]
 * (overwritten).  Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
int splat_pose_rel_grad(int32_t n, const float *w2c, const float *d_cam, float *d_rel, splat_stream_t stream);

/*
 * splat_assoc -- render-based Gaussian association between two maps
 * (Sec. 3.5 step 2): at every pixel where both renders have a maximum-weight
 * Gaussian (id >= 0) and both final transmittances are <= t_max, the pair
 * (id_a, id_b) is formed; the result is the set of distinct pairs in
 * ascending (id_a, id_b) order with the number of pixels of each.
 *   id_a, t_a, id_b, t_b: device [npix]; n_a, n_b: number of Gaussians of
 *   each map (ids must be < n_a, n_b);
 *   pairs: device int32[capacity,2]; counts: device int32[capacity];
 *   m_dev: device int64[1] receives M; status: device int32[1], set to
 *   SPLAT_ECAPACITY when M > capacity (the first `capacity` pairs are kept).
 *   ws: workspace of splat_assoc_workspace_size(npix) bytes.
 * Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
size_t splat_assoc_workspace_size(int64_t npix);
int splat_assoc(const int32_t *id_a, const float *t_a, const int32_t *id_b, const float *t_b,
                int64_t npix, int64_t n_a, int64_t n_b, float t_max, int32_t *pairs,
                int32_t *counts, int64_t capacity, int64_t *m_dev, int32_t *status, void *ws,
                size_t ws_bytes, splat_stream_t stream);

/*
 * splat_loss_consensus -- the inter-agent optimisation loss of Eq. (optim)
 * (Sec. 3.5 step 4) between a rendered image (C, D) and another agent's
 * (C*, D*), with its SSIM term read as w_ssim (1 - SSIM) since the loss is
 * minimised:
 *   L = w_l1 mean|C - C*| + w_ssim (1 - SSIM(C, C*)) + w_geom mean|D - D*|,
 * the paper's weights being 0.8, 0.2, 0.1 (Sec. 4.1).  SSIM is the mean over
 * pixels and channels of the windowed statistic (11 x 11 Gaussian window,
 * sigma 1.5, normalised; the image is zero outside its border;
 * C1 = 0.01^2, C2 = 0.03^2).  Gradients with respect to C and D are written
 * (overwritten) to d_rgb and d_depth (sign(0) = 0); C* and D* get none.
 *   rgb, target_rgb: device float[H,W,3]; depth, target_depth: device float[H,W];
 *   loss: device float[2], ADDED to: loss[0] += L, loss[1] += SSIM (the
 *   caller zeroes it);
 *   ws: splat_loss_consensus_workspace_size(H, W) bytes, 16-byte aligned.
 * Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
size_t splat_loss_consensus_workspace_size(int32_t height, int32_t width);
int splat_loss_consensus(const float *rgb, const float *depth, const float *target_rgb,
                         const float *target_depth, int32_t height, int32_t width, float w_l1,
                         float w_ssim, float w_geom, float *d_rgb, float *d_depth, float *loss,
                         void *ws, size_t ws_bytes, splat_stream_t stream);

/*
 * splat_mahalanobis_system -- the Gauss-Newton system of the inter-agent
 * alignment objective of Sec. 3.5 step 3,
 *   sum_(k,l) w_kl r^T M r,  r = T x_l - x_k,  M^-1 = R Sigma_l R^T + Sigma_k,
 * over associated pairs (k in map A, l in map B; T = (R, t) maps B's world
 * into A's), for the left perturbation T <- exp(delta^) T, delta = (rho, phi).
 * The combined covariance is taken at the current T and held fixed in the
 * step (with R = I it is the printed Sigma_k + Sigma_l).  Sigma = R(q)
 * diag(exp(2 log_scale)) R(q)^T of each Gaussian.
 *   map_a, map_b: the two maps (mean, log_scale, quat are read; quat
 *   16-byte aligned);
 *   pairs: device int32[capacity,2] (8-byte aligned) of (id in A, id in B), as splat_assoc
 *   writes them; weights: device int32[capacity] pair weights (e.g. the pixel
 *   counts of splat_assoc) or NULL for weight 1; m_dev: device int64[1], the
 *   number of valid pairs (min(M, capacity) are used);
 *   T: device float[16] row-major;
 *   max_dist: pairs whose residual |r| at T exceeds it are left out (the
 *   correspondence distance of the G-ICP point selection, 0.02 in Sec. 4.1);
 *   <= 0 keeps every pair;
 *   sys: device double[28], ADDED to (the caller zeroes it): H's upper
 *   triangle row by row (21, H = 2 sum w J^T M J), g (6, g = 2 sum w J^T M r),
 *   cost (1), with J = [I | -[T x_l]x].
 * Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
int splat_mahalanobis_system(const splat_gaussians *map_a, const splat_gaussians *map_b,
                             const int32_t *pairs, const int32_t *weights, const int64_t *m_dev,
                             int64_t capacity, const float *T, float max_dist, double *sys,
                             splat_stream_t stream);

/*
 * splat_mahalanobis_step -- solves H delta = -g of a system written by
 * splat_mahalanobis_system (scaled to unit diagonal, H' = D H D with
 * D = diag(H)^-1/2, then Cholesky in single precision) and applies
 * T <- exp(delta^) T.  delta_out: device double[6] or NULL.  If H is not
 * positive definite T is left unchanged and SPLAT_ENUMERIC is raised in
 * status (device int32[1]).  Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
int splat_mahalanobis_step(const double *sys, float *T, double *delta_out, int32_t *status,
                           splat_stream_t stream);

/*
 * splat_mahalanobis_system_step -- splat_mahalanobis_system followed by
 * splat_mahalanobis_step in one launch: the pairs' contributions are added to
 * sys, and the CTA that finishes last solves the whole accumulated system
 * (including what earlier splat_mahalanobis_system calls added, e.g. other
 * keyframes' pairs), applies T <- exp(delta^) T and sets sys back to zero.
 *   sys: device double[32], 8-byte aligned: the 28 sums as in
 *   splat_mahalanobis_system, then a counter; zero-filled before the first
 *   call, and left zero-filled by every call (no clearing between
 *   iterations).  T: updated in place (read by the pairs' terms first).
 *   delta_out (device double[6] or NULL), status: as splat_mahalanobis_step.
 * Calls on the same sys must not overlap.  Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
int splat_mahalanobis_system_step(const splat_gaussians *map_a, const splat_gaussians *map_b,
                                  const int32_t *pairs, const int32_t *weights, const int64_t *m_dev,
                                  int64_t capacity, float *T, float max_dist, double *sys,
                                  double *delta_out, int32_t *status, splat_stream_t stream);

/*
 * splat_prune -- Gaussian splat pruning (Algorithm 1, Suppl. "Gaussian Splat
 * Pruning for Mapping"): a Gaussian is removed when its opacity
 * 1 / (1 + exp(-logit)) < tau_o, or, when tau_s > 0, when its largest scale
 * exp(log_scale) exceeds tau_s or exceeds tau_e times the sum of the other two
 * (the paper's defaults are 0.005, 0.25, 10).  Every decision is taken in
 * float32 with the exponential of splat_exp_f32 in this order: opacity =
 * 1 / (1 + e), largest = max(max(s0, s1), s2), sum = (s0 + s1) + s2,
 * elongated = largest > tau_e * (sum - largest).
 * The kept rows of every column are written, in their original order, to the
 * column's destination (a column is a float[n, width] array: a parameter, its
 * gradient or an Adam moment), so the map and its optimiser state stay
 * aligned.
 *   g: the map (opacity_logit and log_scale are read);
 *   cols: host array of n_cols (<= 16) descriptors; src and dst must not
 *   overlap; width 1..16;
 *   mask: device uint8[n] (1 = removed) or NULL;
 *   n_keep_dev: device int64[1] receives the number of kept Gaussians;
 *   ws: splat_prune_workspace_size(n) bytes.
 * Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
typedef struct splat_column {
  const float *src;
  float *dst;
  int32_t width;
} splat_column;

size_t splat_prune_workspace_size(int64_t n);
int splat_prune(const splat_gaussians *g, float tau_o, float tau_s, float tau_e,
                const splat_column *cols, int32_t n_cols, uint8_t *mask, int64_t *n_keep_dev,
                void *ws, size_t ws_bytes, splat_stream_t stream);

/*
 * splat_exp_f32 -- the exponential every kernel above uses, over n device
 * floats (exposed so that its agreement with the CPU oracle and its error
 * against the true exp can be tested).  Cody & Waite range reduction with a
 * two-part ln 2, degree-7 Taylor polynomial, scaling by 2^k; x > 88 -> inf,
 * x < -87 -> 0.  Errors: SPLAT_EINVAL, SPLAT_ECUDA.
 */
int splat_exp_f32(const float *x, float *y, int64_t n, splat_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* SPLAT_H */
