/*
 * mvs.h -- C ABI of the GB300 PatchMatch multi-view-stereo library
 * (depth-map path of PHI-MVS, Sun et al., arXiv 2104.06165).
 *
 * The library estimates, for every pixel x of a reference image, a depth d_x
 * and a unit normal n_x (Sec. III: "estimate depth and normal values for each
 * pixel on each reference image") from images and calibrated cameras
 * (Sec. I: "3D structure using 2D images and camera parameters").
 *
 * General rules
 *   - Every entry point returns an mvs_status; nothing throws or aborts across
 *     the ABI.  On failure the context keeps a message (mvs_last_error).
 *   - One context is used by one host thread at a time.
 *   - All GPU work is ordered on the context's CUDA stream (the stream given
 *     to mvs_create).  Calls whose outputs are device pointers return after
 *     enqueueing; calls with host outputs synchronise that stream.
 *   - Arrays are row-major; pixel (x, y) of a W x H view is element y*W + x.
 *     Pixel centres sit at integer coordinates.
 *   - Device pointers must be allocated on the context's device; the caller
 *     owns every buffer it passes.  The library owns its context memory.
 *   - Plane maps hold 4 floats per pixel: (n.x, n.y, n.z, depth) with the
 *     normal in the reference camera frame facing the camera
 *     (n . K^-1 (x, y, 1) < 0) and depth the camera z-depth; depth 0 marks a
 *     pixel without a depth.
 */
#ifndef MVS_H
#define MVS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MVS_OK = 0,
    MVS_EINVAL = 1,       /* bad argument (NULL pointer, size, index, range) */
    MVS_ENOMEM = 2,       /* device or host allocation failed               */
    MVS_ECUDA = 3,        /* a CUDA call failed (message has the CUDA error) */
    MVS_ETIMEOUT = 4,     /* a bounded device wait ran out                   */
    MVS_ESTATE = 5,       /* a needed depth map was never computed           */
    MVS_EUNSUPPORTED = 6  /* parameter combination not built                 */
} mvs_status;

/* Calibrated pinhole camera: x_cam = R * X_world + t, pixel = K * x_cam. */
typedef struct {
    double K[9];          /* row-major intrinsics, last row (0, 0, 1)        */
    double R[9];          /* row-major rotation world -> camera              */
    double t[3];
    int32_t width, height;
} mvs_camera;

typedef struct mvs_ctx mvs_ctx;   /* opaque, owned by the library */

enum { MVS_MEM_DEVICE = 0, MVS_MEM_HOST = 1 };
enum { MVS_INIT_RANDOM = 0,       /* Sec. III-B random initialisation        */
       MVS_INIT_GIVEN = 1,        /* start from out->plane and out->cost     */
       MVS_INIT_GIVEN_RECOST = 2, /* start from out->plane, compute its cost */
       MVS_INIT_RANGE = 3         /* Sec. III-B with per-pixel depth ranges
                                     from sparse features (init_range)       */
};

/* PatchMatch parameters (Sec. III-B, III-C; defaults in Sec. IV). */
typedef struct {
    float win_radius;      /* r_orig: half side of the matching window, px   */
    int32_t win_samples;   /* samples per axis n = 2 r_now + 1 (2..22); the
                              offsets are s*k, k = -r_now..r_now, s = r_orig /
                              r_now (Sec. III-C, dilated window)             */
    float sigma_s;         /* bilateral spatial sigma in px; <= 0: none      */
    float sigma_c;         /* bilateral colour sigma on the [0,1] intensity
                              scale; <= 0 together with sigma_s <= 0 gives
                              the unweighted ZNCC of Eq. 4                   */
    float d_lo, d_hi;      /* depth range of initialisation / refinement    */
    int32_t iters;         /* iterations (one = red phase + black phase)     */
    int32_t phase_begin;   /* first half-iteration to run (0 = red of it. 0) */
    int32_t phase_end;     /* one past the last half-iteration; < 0 means
                              2 * iters                                      */
    int32_t init_mode;     /* MVS_INIT_*                                     */
    uint64_t seed;         /* Philox4x64-10 key word 0 (word 1 = ref index)  */
    int32_t precision;     /* 0 = FP32; 1 = mixed: the bilinear interpolation
                              of two window samples per half2 instruction on
                              intensities shifted by an intensity of the
                              source patch, moments in FP32, near-flat
                              variance denominators recomputed in FP64
                              (results differ from FP32 by the fp16 rounding
                              of the interpolated values)                    */
    int32_t lanes_per_pixel; /* work layout of the ZNCC kernels: lanes that
                              share one window (4, 8, 16 or 32; 0 = default;
                              -1 = timed choice, mvs_patchmatch_batch only).
                              Results are identical for every choice up to
                              float rounding of the group reductions.        */
    int32_t n_prop;        /* learned proposals per pixel, 0..8 (0: none)    */
    int32_t reserved0;
    const float* proposals;/* DEVICE, H*W*n_prop*4 (n.x, n.y, n.z, depth)
                              planes per pixel, e.g. from mvs_propose; in
                              every half-iteration each pixel of the phase's
                              colour scores its n_prop proposals right after
                              the propagated planes and takes the cheapest
                              if it is strictly cheaper than its state (no
                              counterpart in the paper: extra candidates of
                              the propagation step, judged by Eq. 5).  Zero
                              depth marks an unused slot.  NULL with
                              n_prop = 0.                                    */
    const float* init_range;/* DEVICE, H*W*2 (d_min, d_max) per pixel for
                              init_mode MVS_INIT_RANGE, e.g. from
                              mvs_sparse_depth_range: the initial depth is
                              d_min + (d_max - d_min) u with the Philox draw u
                              of the random initialisation; NaN: the whole
                              range [d_lo, d_hi].  8-byte aligned.  NULL for
                              the other modes.  mvs_patchmatch_batch: the
                              ranges of all refs back to back, in refs
                              order.                                         */
} mvs_pm_params;

/* Depth-map buffers supplied by the caller. */
typedef struct {
    float* plane;          /* H*W*4: (n.x, n.y, n.z, depth)                  */
    float* cost;           /* H*W aggregated cost C(x) of Eq. 5              */
    int32_t mem;           /* MVS_MEM_DEVICE or MVS_MEM_HOST                 */
} mvs_depth_map;

/* Geometric-consistency filter parameters (Sec. III-D). */
typedef struct {
    float depth_tol;       /* 0.02                                           */
    int32_t depth_relative;/* 0: |d_j(x'_j) - z_j(X)| (paper); 1: relative   */
    float max_angle_deg;   /* 30                                             */
    float max_reproj_px;   /* 1                                              */
    int32_t min_consistent;/* "more than one" consistent view: 2             */
} mvs_filter_params;

/* Plane hypothesis inference parameters (Sec. III-E, Sec. IV). */
typedef struct {
    float kappa1, kappa2, kappa3;  /* Eq. 6 / Eq. 7: 4, 0.5, 2               */
    int32_t n_fit;         /* closest reconstructed pixels per line fit: 6   */
    int32_t fit_inverse;   /* 0: fit depth (paper); 1: fit 1/depth           */
    int32_t trw_iters;     /* TRW iterations (forward + backward pass): 1    */
    float hole_cost;       /* with keep_mask == NULL, pixels whose stored
                              cost >= hole_cost (or without depth) are holes */
    int32_t selection;     /* MVS_PHI_SELECT_MRF (0, the paper's PHI-MVS) or
                              MVS_PHI_SELECT_MIN_COST (1, PHI-MVS/M of
                              Sec. IV, Table I: no MRF, each hole takes its
                              valid hypothesis of minimal matching cost)    */
} mvs_phi_params;

enum { MVS_PHI_SELECT_MRF = 0, MVS_PHI_SELECT_MIN_COST = 1 };

/* ------------------------------------------------------------------------ */

/* Create a context and copy the images to the device.
 *   cams[n_views], images[n_views]: host pointers to uint8 grayscale images of
 *   cams[i].width x cams[i].height, pitch = width.  The images are copied (the
 *   caller keeps its buffers).  cuda_stream: a cudaStream_t or NULL for the
 *   legacy default stream.  The context uses the current CUDA device.
 * Errors: MVS_EINVAL (NULL pointers, n_views < 2, width or height < 2 or > 32768),
 *   MVS_ENOMEM, MVS_ECUDA. */
mvs_status mvs_create(const mvs_camera* cams, const uint8_t* const* images, int32_t n_views,
                      void* cuda_stream, mvs_ctx** out);

/* Release everything the context owns.  NULL-safe.  Synchronises its stream. */
void mvs_destroy(mvs_ctx* ctx);

/* Message of the last failed call on ctx (or of the last failed mvs_create
 * when ctx is NULL); valid until the next call on ctx. */
const char* mvs_last_error(const mvs_ctx* ctx);

/* Depth and normal map of reference view `ref` from source views srcs[n_src]
 * by checkerboard PatchMatch (Sec. III-B random init, Sec. III-C Eq. 4 ZNCC
 * with dilated window and plane-induced homography, Eq. 5 aggregation, red-
 * black propagation and four-candidate random refinement).
 *   Runs half-iterations [phase_begin, phase_end) after the initialisation
 *   chosen by init_mode; the counter-based random numbers make a run split
 *   into several calls (MVS_INIT_GIVEN) identical to one uninterrupted run.
 *   out: caller buffers of the reference's size; with MVS_INIT_GIVEN* they
 *   also carry the starting state.  The result is kept in the context for
 *   mvs_geo_filter / mvs_plane_infer.
 * Errors: MVS_EINVAL (bad index, duplicate or self source, n_src outside
 *   1..32, window outside 2..22 samples, d_lo >= d_hi, NULL buffers),
 *   MVS_EUNSUPPORTED (precision other than 0 or 1), MVS_ENOMEM, MVS_ECUDA. */
mvs_status mvs_patchmatch(mvs_ctx* ctx, int32_t ref, const int32_t* srcs, int32_t n_src,
                          const mvs_pm_params* params, mvs_depth_map* out);

/* Depth maps of several reference views in one call: for each view in
 * turn, its initialisation and its half-iterations in the phase range
 * (Algorithm 1 loops over reference images; the views are independent, so
 * the results equal those of separate mvs_patchmatch calls).  The kernels
 * are captured into a CUDA graph on the first call with a given
 * (refs, srcs, params) and the graph is replayed by later calls.
 *   refs[n_ref]: reference views (distinct); srcs[n_ref * n_src]: row r holds
 *   the n_src sources of refs[r]; outs[n_ref]: depth-map buffers of each
 *   reference's size, all in the same memory kind.  params as for
 *   mvs_patchmatch; params->lanes_per_pixel = -1 asks the library to time
 *   the work layouts on the first call (two iterations of the first view,
 *   each from the same initial state, in the view's own buffers before its
 *   real run) and keep the fastest for this window size.  With
 *   MVS_INIT_RANGE, params->init_range holds the ranges of every reference
 *   back to back in refs order (sum of H*W*2 floats); with n_prop > 0,
 *   params->proposals likewise holds every reference's proposals back to
 *   back (sum of H*W*n_prop*4 floats).  The graph is keyed by the params,
 *   so the buffers behind init_range and proposals must keep their address
 *   between the calls that replay it.
 *   The maps stay in the context for mvs_geo_filter.
 * Errors: as mvs_patchmatch, plus MVS_EINVAL for n_ref < 1 or repeated refs. */
mvs_status mvs_patchmatch_batch(mvs_ctx* ctx, int32_t n_ref, const int32_t* refs, const int32_t* srcs,
                                int32_t n_src, const mvs_pm_params* params, mvs_depth_map* outs);

/* Store a depth map of `view` that was computed elsewhere (another
 * process or GPU, after the exchange before the geometric filter) in the
 * context, as mvs_patchmatch would have left it, for mvs_geo_filter,
 * mvs_fuse and mvs_plane_infer (no counterpart in the paper).
 *   plane: H*W*4 floats (n.x, n.y, n.z, depth; depth 0 = none), cost: H*W
 *   floats or NULL (then the stored costs are C_max = 2); both in `mem`,
 *   plane 16-byte and cost 4-byte aligned.  Copied; the caller keeps its
 *   buffers.  Stream-ordered (synchronises for host buffers).
 * Errors: MVS_EINVAL (bad view, NULL plane, alignment, mem kind),
 *   MVS_ENOMEM, MVS_ECUDA. */
mvs_status mvs_set_depth_map(mvs_ctx* ctx, int32_t view, const float* plane, const float* cost, int32_t mem);

/* Aggregated cost (Eq. 4/5) of a given plane map of view `ref`.
 *   plane: H*W*4 input, cost: H*W output, view_cost: H*W*n_src output of the
 *   per-view costs C(x, j) (C_max = 2 for an excluded view) or NULL.  All
 *   three live in `mem` (device or host).
 * Errors as mvs_patchmatch. */
mvs_status mvs_plane_cost(mvs_ctx* ctx, int32_t ref, const int32_t* srcs, int32_t n_src,
                          const mvs_pm_params* params, const float* plane, float* cost, float* view_cost,
                          int32_t mem);

/* Geometric-consistency filter of view `ref` against srcs (Sec. III-D):
 *   keep_mask[H*W] (in `mem`) receives 1 for pixels consistent with at least
 *   min_consistent source maps, else 0; count (H*W int32, may be NULL)
 *   receives the number of consistent views.
 * Errors: MVS_ESTATE if ref or a source has no depth map in the context,
 *   MVS_EINVAL, MVS_ECUDA. */
mvs_status mvs_geo_filter(mvs_ctx* ctx, int32_t ref, const int32_t* srcs, int32_t n_src,
                          const mvs_filter_params* fp, uint8_t* keep_mask, int32_t* count, int32_t mem);

/* Depth-map fusion into one point cloud (Sec. III-F, the last step of
 * Algorithm 1).  The views are taken in the order given; every remaining
 * pixel x of image i (depth > 0, kept by its mask, not merged before) is
 * back-projected to X_i, and for every later image j the pixel [x'_j] that
 * X_i projects to (nearest pixel) is back-projected to X'_j; when
 * |X_i - X'_j| < rel_tol * (z-depth of X_i in image i) that pixel is merged:
 * removed from image j, X'_j joins the average.  The paper fixes no
 * precision; the decisions are taken in single precision, every operation
 * rounded on its own, in the order stated in fuse_kernels.cu (readings:
 * pinhole K, the distance relative to the z-depth, nearest pixel by
 * floor(u + 1/2)).
 *   views[n_views]: processing order, distinct views whose depth maps are in
 *   the context (mvs_patchmatch / mvs_plane_infer results).
 *   keep_masks: NULL, or n_views pointers to H*W uint8 masks (1 = kept) or
 *   NULL (every pixel with depth); masks live in `mem`.
 *   rel_tol: the paper's 0.01.
 *   points: capacity x 4 floats (x, y, z, merged pixel count) in world
 *   coordinates, written in processing order of the views, then raster order
 *   of the emitting pixel; src: capacity x 2 int32 (view, pixel index) or
 *   NULL; owner: NULL, or one int64 per pixel of the views, view after view
 *   in processing order, raster order within a view: the index of the point
 *   the pixel went into (emitted or merged), -1 for a pixel that was never
 *   present (no depth or not kept); all in `mem` (device or host).  The call
 *   synchronises and sets *n_points to the number of points of the cloud.
 * Errors: MVS_EINVAL (bad or repeated view, rel_tol <= 0, bad buffers, or
 *   more points than capacity: then the first `capacity` points are written
 *   and *n_points holds the full count), MVS_ESTATE (a view without depth
 *   map), MVS_EUNSUPPORTED (a view whose K is not pinhole), MVS_ENOMEM,
 *   MVS_ECUDA. */
mvs_status mvs_fuse(mvs_ctx* ctx, int32_t n_views, const int32_t* views, const uint8_t* const* keep_masks,
                    float rel_tol, float* points, int32_t* src, int64_t* owner, int64_t capacity,
                    int64_t* n_points, int32_t mem);

/* Neighbouring-image selection (Sec. III-A, Eqs. 1-3) for every view of the
 * context (2..64 views), from sparse 3D points of a structure-from-motion
 * step.  For reference i and source j, A = the points visible in both;
 * Eq. 1 disturbs X in A to (1 + eps) X - eps C_i; Eq. 2 gives tau = mean
 * |x^'_j - x'_j| (pixels); sources with tau < t_tau or no shared point are
 * removed and the rest sorted by Eq. 3's zeta = min(b_ij, 0.1)
 * min(theta_ij, 0.05) / N_A (b: baseline, theta: angle between the
 * principal axes in radians; tie: lower index).  FP64 throughout.
 *   points: n_points x 3 doubles (world); vis: n_points masks, bit v set when
 *   the point is visible in view v; eps, t_tau: the disturbance and the
 *   threshold in pixels (Sec. IV uses eps = 0.002 and t_tau = 0.1:
 *   MVS_NBR_EPS, MVS_NBR_T_TAU); k: neighbours per view (the paper keeps 8).
 *   neighbors: n_views x k int32, the selected sources per view in order,
 *   -1 past the kept ones; tau / zeta (n_views x n_views doubles, zeta +inf
 *   for removed sources) and n_shared (n_views x n_views int32) may be NULL.
 *   All buffers in `mem`.  The call synchronises.
 * Errors: MVS_EINVAL (view count, k outside 1..n_views-1, eps <= 0, t_tau < 0,
 *   NULL buffers), MVS_ENOMEM, MVS_ECUDA. */
#define MVS_NBR_EPS 0.002   /* Eq. 1's disturbance, Sec. IV */
#define MVS_NBR_T_TAU 0.1   /* Eq. 2's threshold in pixels, Sec. IV */
mvs_status mvs_select_neighbors(mvs_ctx* ctx, int64_t n_points, const double* points, const uint64_t* vis,
                                double eps, double t_tau, int32_t k, int32_t* neighbors, double* tau,
                                int32_t* n_shared, double* zeta, int32_t mem);

/* Per-pixel depth ranges for the initialisation from sparse features
 * (Sec. III-B) of view `ref`.  Features: the sparse points visible in ref
 * whose re-projection error is below max_reproj (the paper's 2) and that
 * are visible in at least floor(v - 1) images, v the mean number of images
 * per point; each keeps its observation in ref and its z-depth there.  Per
 * pixel, the closest feature in each of the four quadrants around it within
 * W / 10 pixels gives [d_min, d_max] over those features, clamped to
 * [d_lo, d_hi]; NaN where no feature is that close.  The closest-feature
 * choice is taken in single precision, every operation rounded on its own,
 * the first point winning a tie.
 *   points: n_points x 3 doubles (world); vis: n_points masks (bit v:
 *   visible in view v); reproj: n_points doubles; obs: n_points x 2 doubles,
 *   the observation of each point in view ref (any value where not visible);
 *   range: H*W*2 floats (d_min, d_max) out.  All in `mem`.  The call
 *   synchronises when mem is MVS_MEM_HOST.
 * Errors: MVS_EINVAL (bad view, NULL buffers, d_lo >= d_hi, more than 64
 *   views), MVS_ENOMEM, MVS_ECUDA. */
mvs_status mvs_sparse_depth_range(mvs_ctx* ctx, int32_t ref, int64_t n_points, const double* points,
                                  const uint64_t* vis, const double* reproj, const double* obs, double max_reproj,
                                  float d_lo, float d_hi, float* range, int32_t mem);

/* Plane hypothesis inference (Sec. III-E) on view `ref`: four line-fit
 * hypotheses per hole, their matching cost through the sources, a pairwise
 * MRF (Eq. 6-9) decoded by TRW at half resolution, closest-hypothesis
 * selection, Eq. 10 normals (phi->selection = MVS_PHI_SELECT_MIN_COST: the
 * minimal-cost hypothesis per hole in place of the MRF and its selection).
 *   keep_mask[H*W] (in `mem`): 1 = reconstructed; NULL derives holes from
 *   the stored cost (cost >= hole_cost or no depth).  inout: the depth map
 *   (MVS_INIT_GIVEN state of the view); on return holes that were filled
 *   carry their plane, remaining holes and dropped pixels have depth 0.  The
 *   context's copy of the view is updated.  pm gives the window / ZNCC
 *   parameters for the hypothesis costs.
 * Errors: MVS_ESTATE if the view has no depth map, MVS_EINVAL (also for an
 *   unknown selection), MVS_ECUDA. */
mvs_status mvs_plane_infer(mvs_ctx* ctx, int32_t ref, const int32_t* srcs, int32_t n_src,
                           const mvs_pm_params* pm, const mvs_phi_params* phi, const uint8_t* keep_mask,
                           mvs_depth_map* inout);

/* Stages of mvs_plane_infer, exposed for stage-by-stage checking.
 * All buffers are in `mem`.
 *  mvs_phi_hypotheses: depth[H*W] and known[H*W] (1 = reconstructed) ->
 *    hyp[H*W*4] depths of the four directions (horizontal, vertical, 45 deg
 *    below, 45 deg above), valid[H*W*4] flags.
 *  mvs_phi_cost: hypothesis depths -> hcost[H*W*4] (Eq. 5 cost of the
 *    fronto-parallel plane at that depth, C_max where invalid).
 *  mvs_phi_mrf: half-resolution MRF from (known, depth, hyp, valid, hcost) ->
 *    label[gh*gw] (chosen hypothesis index 0..3, -1 for a reconstructed node,
 *    -2 for a node without labels), gw = (W+1)/2, gh = (H+1)/2.
 *  mvs_phi_select: labels -> plane[H*W*4] filled with the closest hypothesis
 *    and its Eq. 10 normal (known pixels keep their plane).
 *  mvs_phi_select_min_cost: the selection of PHI-MVS/M (Sec. IV, Table I)
 *    in place of mvs_phi_mrf + mvs_phi_select: each hole takes its valid
 *    hypothesis of minimal hcost (the lowest index on a tie), then its
 *    Eq. 10 normal; a hole without a valid hypothesis, or without four
 *    neighbours with depth, is zeroed.  hyp and hcost 16-byte, valid 4-byte
 *    aligned. */
mvs_status mvs_phi_hypotheses(mvs_ctx* ctx, int32_t W, int32_t H, const float* depth, const uint8_t* known,
                              const mvs_phi_params* phi, float d_lo, float d_hi, float* hyp, uint8_t* valid,
                              int32_t mem);
mvs_status mvs_phi_cost(mvs_ctx* ctx, int32_t ref, const int32_t* srcs, int32_t n_src,
                        const mvs_pm_params* pm, const float* hyp, const uint8_t* valid, float* hcost,
                        int32_t mem);
mvs_status mvs_phi_mrf(mvs_ctx* ctx, int32_t W, int32_t H, const uint8_t* known, const float* depth,
                       const float* hyp, const uint8_t* valid, const float* hcost, const mvs_phi_params* phi,
                       int32_t* label, int32_t mem);
mvs_status mvs_phi_select(mvs_ctx* ctx, int32_t ref, const uint8_t* known, const float* hyp,
                          const uint8_t* valid, const int32_t* label, float* plane, int32_t mem);
mvs_status mvs_phi_select_min_cost(mvs_ctx* ctx, int32_t ref, const uint8_t* known, const float* hyp,
                                   const uint8_t* valid, const float* hcost, float* plane, int32_t mem);

/* Allocation-free variant of mvs_phi_hypotheses (the paper has no
 * counterpart; this is a deployment convenience).
 *   Some callers cannot allocate device memory once they are running: a
 *   service that reserves its whole device-memory budget at start-up and
 *   treats any later cudaMalloc as a fault, an engine whose own allocator owns
 *   every byte of the device, or a latency-bound pipeline that cannot afford
 *   the device-wide synchronisation cudaMalloc / cudaFree imply.  This entry
 *   point computes exactly what mvs_phi_hypotheses computes but keeps its
 *   line-gap scratch in a fixed array compiled into the library
 *   (MVS_PHI_STATIC_MAX_PIXELS pixels x 32 bytes = 8 MiB per device, held by
 *   every device that loads the library until the process exits), so it
 *   calls no cudaMalloc, cudaFree or allocating library routine.
 *   depth, known, hyp, valid: DEVICE pointers only (layout as in
 *   mvs_phi_hypotheses); work is enqueued on the context stream.
 *   The first call on a device looks up the array's device address (with
 *   that device current); make that first call before any stream capture.
 *   Every call shares the one array: calls that overlap on the GPU (other
 *   streams, other contexts, other threads) race and must be serialised by
 *   the caller.  Every entry a call reads is written by the same call first,
 *   so no clearing is needed between calls.
 * Errors: MVS_EINVAL (NULL argument, W*H > MVS_PHI_STATIC_MAX_PIXELS, bad
 *   size or n_fit), MVS_ECUDA. */
#define MVS_PHI_STATIC_MAX_PIXELS 262144
mvs_status mvs_phi_hypotheses_static(mvs_ctx* ctx, int32_t W, int32_t H, const float* depth,
                                     const uint8_t* known, const mvs_phi_params* phi, float d_lo, float d_hi,
                                     float* hyp, uint8_t* valid);

/* Measurement hooks (no counterpart in the paper).
 *  mvs_profile(ctx, enable): enable != 0 makes mvs_patchmatch bracket every
 *    checkerboard-phase kernel with CUDA events on the context stream; any
 *    call resets the accumulated figures.
 *  mvs_profile_read: synchronises the context stream and returns the summed
 *    event time of the phase kernels in ms and their number since the last
 *    reset, the number of kernels the library launched (all contexts) since
 *    the last reset, and the number of (pixel, hypothesis, source view) ZNCC
 *    evaluations the phase kernels performed (views whose window left the
 *    source image and pixels with a flat reference patch are not evaluated).
 *    Any of the pointers may be NULL.
 * Errors: MVS_EINVAL for a NULL ctx, MVS_ECUDA. */
mvs_status mvs_profile(mvs_ctx* ctx, int32_t enable);
mvs_status mvs_profile_read(mvs_ctx* ctx, double* phase_ms, int64_t* phase_launches, int64_t* kernel_launches,
                            int64_t* phase_evals);

/* Measured peaks of device `device` for the roofline of the PatchMatch
 * kernels (no counterpart in the paper), each the fastest of five timed
 * launches after a warm-up launch of a small kernel of this library:
 *   fp32_flops: FP32 FMA rate (flop/s, FMA = 2) of 16 independent chains per
 *     thread on every SM;
 *   gathers: 8-byte loads per second served from L1 in the window-sample
 *     pattern of the phase kernel (two groups of 16 lanes per warp, texels
 *     two apart, eight independent loads in flight per thread);
 *   l2_bytes: read bandwidth (bytes/s) of a 64 MB buffer resident in L2.
 * Figures depend on the clocks of the moment; callers sample them.  Any
 * output may be NULL (not measured).  Allocates and frees its own device
 * buffers (about 70 MB) and synchronises.
 * Errors: MVS_EINVAL (bad device, all outputs NULL), MVS_ENOMEM, MVS_ECUDA. */
mvs_status mvs_measure_peaks(int32_t device, double* fp32_flops, double* gathers, double* l2_bytes);

/* ------------------------------------------------------------------------
 * Learned plane proposals (no counterpart in the paper).
 *
 * A small U-Net maps a PatchMatch state of a reference view (image, plane
 * map, cost map after one or two iterations) to K = 4 planes per pixel that
 * mvs_patchmatch then scores as extra propagation candidates
 * (mvs_pm_params.n_prop / proposals); the Eq. 5 cost still decides, so a
 * bad proposal is never taken over a better plane.
 *
 * Network: 16 input channels (image / 255, inverse depth normalised to
 * [1/d_hi, 1/d_lo] -> [0, 1], normal (3), cost / 2, ten zero channels);
 * encoder 3x3 conv + ReLU at 32, 48, 64, 96, 128 channels with 2x2 average
 * pooling between levels; decoder nearest 2x up-sampling, concatenation
 * with the encoder output of the level, 3x3 conv + ReLU at 96, 64, 48, 32
 * channels; 1x1 head to 16 outputs = 4 x (a, m.x, m.y, m.z).  Proposal k
 * has inverse depth 1/d_hi + (1/d_lo - 1/d_hi) sigmoid(a_k) and normal
 * m_k / |m_k| turned to face the camera.  Weights and activations are
 * bfloat16 with fp32 accumulation; master weights and Adam moments fp32.
 * Parameters are ordered layer by layer (e0..e4, d3..d0, head), each as
 * weights [c_out][tap][c_in] (tap = 3 dy + dx of the 3x3 stencil) then
 * bias [c_out].
 *
 * Training loss over the pixels with mask != 0:
 *   L = 1/(W H) sum_x min_k ( |rho_k - 1/d_t| / (1/d_lo - 1/d_hi)
 *                             + lambda (1 - |n_k . n_t|) ),  lambda = 0.1
 * (first k on ties), targets (n_t, d_t) a plane map.
 *
 * All image, map and output pointers below are DEVICE pointers on the
 * network's device; W and H are multiples of 16 within the capacity given
 * to mvs_cnn_create.  Work is ordered on the stream given there.
 * ------------------------------------------------------------------------ */
typedef struct mvs_cnn mvs_cnn;   /* opaque, owned by the library */

/* Create a network for images up to max_width x max_height (multiples of 16,
 * at most 8192) and depth range [d_lo, d_hi], with He-initialised weights
 * drawn from `seed`; buffers for activations and gradients at the maximum
 * size are allocated here (about 2.3 kB per pixel).
 * Errors: MVS_EINVAL, MVS_ENOMEM, MVS_ECUDA. */
mvs_status mvs_cnn_create(int32_t max_width, int32_t max_height, float d_lo, float d_hi, uint64_t seed,
                          void* cuda_stream, mvs_cnn** out);
void mvs_cnn_destroy(mvs_cnn* net);              /* NULL-safe */
const char* mvs_cnn_last_error(const mvs_cnn* net);

/* Number of parameters (weights and biases of all layers). */
mvs_status mvs_cnn_n_params(const mvs_cnn* net, int64_t* count);
/* Copy all parameters, or the gradients of the last mvs_cnn_backward, to a
 * HOST array of mvs_cnn_n_params floats, or set the parameters from one
 * (the bfloat16 copies are refreshed).  These synchronise the stream. */
mvs_status mvs_cnn_get_params(mvs_cnn* net, float* host_out);
mvs_status mvs_cnn_set_params(mvs_cnn* net, const float* host_in);
mvs_status mvs_cnn_get_grads(mvs_cnn* net, float* host_out);

/* Forward pass: img[H*W] uint8, plane[H*W*4], cost[H*W] -> out[H*W*16] raw
 * head outputs (fp32). */
mvs_status mvs_cnn_forward(mvs_cnn* net, const uint8_t* img, const float* plane, const float* cost, int32_t W,
                           int32_t H, float* out);

/* Forward pass, loss against target[H*W*4] (planes) on mask[H*W] != 0 and
 * backward pass; the gradients replace those of the previous call.  W is at
 * most 768 here.  loss_out: HOST float or NULL (non-NULL synchronises). */
mvs_status mvs_cnn_backward(mvs_cnn* net, const uint8_t* img, const float* plane, const float* cost, int32_t W,
                            int32_t H, const float* target, const uint8_t* mask, float* loss_out);

/* Stored tensors of the last mvs_cnn_forward / mvs_cnn_backward, for
 * layer-by-layer checking (no counterpart in the paper).  Channels-last
 * bfloat16 (raw 16-bit words), except MVS_CNN_T_HEAD (fp32), at the size of
 * the last call: level l holds (W >> l) x (H >> l) pixels.
 *   MVS_CNN_T_INPUT       level 0, 16 channels (network input)
 *   MVS_CNN_T_ENC         e_l, l = 0..4 (32, 48, 64, 96, 128 channels)
 *   MVS_CNN_T_POOL        avgpool2(e_l) at level l + 1, l = 0..3
 *   MVS_CNN_T_CAT         [up2(d_{l+1} or e_4) | e_l], l = 0..3
 *                         (224, 160, 112, 80 channels for l = 3..0)
 *   MVS_CNN_T_DEC         d_l, l = 0..3 (32, 48, 64, 96 channels)
 *   MVS_CNN_T_HEAD        head output, level 0, 16 fp32 channels
 *   MVS_CNN_T_GRAD_HEAD   d loss / d head output rounded to bf16
 *   MVS_CNN_T_GRAD_DEC    d loss / d (pre-ReLU) d_l, l = 0..3
 *   MVS_CNN_T_GRAD_CAT    d loss / d cat_l, l = 0..3
 *   MVS_CNN_T_GRAD_ENC    d loss / d (pre-ReLU) e_l, l = 0..4
 *   MVS_CNN_T_GRAD_POOL   d loss / d pool_l (before the pooling's backward)
 * host_out receives `bytes` bytes, which must equal the tensor's size.
 * The call synchronises.  Errors: MVS_EINVAL (no such tensor, size
 * mismatch, no call yet), MVS_ECUDA. */
enum {
    MVS_CNN_T_INPUT = 0, MVS_CNN_T_ENC = 1, MVS_CNN_T_POOL = 2, MVS_CNN_T_CAT = 3, MVS_CNN_T_DEC = 4,
    MVS_CNN_T_HEAD = 5, MVS_CNN_T_GRAD_HEAD = 6, MVS_CNN_T_GRAD_DEC = 7, MVS_CNN_T_GRAD_CAT = 8,
    MVS_CNN_T_GRAD_ENC = 9, MVS_CNN_T_GRAD_POOL = 10
};
mvs_status mvs_cnn_read(mvs_cnn* net, int32_t tensor, int32_t level, void* host_out, int64_t bytes);

/* The convolutions wait on their operand copies and tensor-core products
 * through mbarriers with a bound of about a second; a wait that runs out
 * makes the kernel give up (after draining what it issued) and the next
 * call on `net` that synchronises (get_params, get_grads, set_params,
 * backward with loss_out, read, test_timeout) returns MVS_ETIMEOUT once.
 * mvs_cnn_test_timeout runs one small convolution whose first wait targets
 * a barrier that nothing completes, with a wait limit of about 0.1 ms, and
 * returns what that reports (MVS_ETIMEOUT): a check of the path, no
 * counterpart in the paper.  It overwrites the first encoder activations. */
mvs_status mvs_cnn_test_timeout(mvs_cnn* net);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with
 * learning rate lr on the gradients of the last mvs_cnn_backward. */
mvs_status mvs_cnn_adam_step(mvs_cnn* net, float lr);

/* Forward pass and decoding: proposals[H*W*4*4] = 4 planes per pixel
 * (n.x, n.y, n.z, depth) for the reference camera with inverse intrinsics
 * Kinv (host, row-major). */
mvs_status mvs_cnn_propose(mvs_cnn* net, const uint8_t* img, const float* plane, const float* cost, int32_t W,
                           int32_t H, const double Kinv[9], float* proposals);

/* mvs_cnn_propose on the image and the current depth map of context view
 * `ref` (the state left by the last mvs_patchmatch of that view); runs on
 * the context stream, which must be the network's device.
 * Errors: MVS_ESTATE if the view has no map, MVS_EINVAL, MVS_ECUDA. */
mvs_status mvs_propose(mvs_ctx* ctx, int32_t ref, mvs_cnn* net, float* proposals);

#ifdef __cplusplus
}
#endif
#endif /* MVS_H */
