/*
 * vgicp.h -- C ABI of the B300 voxelised-GICP factor library.
 *
 * Operations (Koide et al., "Globally Consistent 3D LiDAR Mapping with
 * GPU-accelerated GICP Matching Cost Factors", RA-L 2021):
 *   - voxelmap build: Sec. III-A, voxel data association (a voxel holds the
 *     mean of its points' means and the mean of their covariances);
 *   - factor linearisation: Eq. 1-6 (cost, 12x12 Gauss-Newton H, 12-vector b);
 *   - overlap: Eq. 7-8;
 *   - per-point covariance estimation from k neighbours: Sec. III (overview).
 *
 * Conventions used by every call:
 *   - Poses are 12 doubles, row-major 3x4 [R | t], world-from-frame.
 *   - A factor has a target B (owner of the voxelmap) and a source A (whose
 *     points are summed over); source points are mapped into the target frame
 *     by T_BA = T_B^-1 T_A, computed in float64 as
 *     R_BA[i][j] = sum_k R_B[k][i] R_A[k][j], t_BA[i] = sum_k R_B[k][i] (t_A[k] - t_B[k]),
 *     k = 0, 1, 2, every product and sum separately rounded.
 *   - Tangent: right perturbation T <- T Exp(xi), xi = (omega, v), rotation
 *     first; the 12-vector is [xi_B ; xi_A].  H is the full symmetric 12x12
 *     matrix, row-major, H = sum J^T Omega J, b = sum J^T Omega e, cost =
 *     sum e^T Omega e with e = mu_B - T_BA p and Omega = (C_B + R C_A R^T)^-1
 *     (no factor 1/2, no weighting by voxel point count).
 *   - Voxel coordinate of a point x (target frame): k = floor(x * (1/r)),
 *     x formed in float64 as fma(R0, px, fma(R1, py, fma(R2, pz, t))); valid
 *     iff -2^20 <= k <= 2^20 - 1 on every axis and x is finite.  A source point
 *     corresponds to the one target voxel containing it, or to none.
 *   - Points: n x 3 float32 (x, y, z).  Covariances: n x 6 float32
 *     (c00, c01, c02, c11, c12, c22), symmetric positive definite.
 *
 * Memory: mem_kind / out_kind say where a caller pointer lives.  HOST
 * pointers may be pageable; DEVICE inputs are read by work enqueued on the
 * context's current lane (copied into library-owned device memory there), so
 * they must stay valid and unchanged until that lane has been synchronised
 * (vgicp_synchronize, or any later call with HOST outputs on the same lane).
 * HOST inputs in pageable memory (and any below 64 KB) are staged
 * before the call returns, so the caller may reuse them at once; HOST inputs in
 * page-locked memory of 64 KB or more are copied by the device in stream order,
 * like cudaMemcpyAsync: leave them unchanged until the lane has been
 * synchronised (vgicp_synchronize, or any later call with HOST outputs on the
 * same lane).  Handles own their device memory until vgicp_release() or
 * vgicp_destroy().  Output buffers are always caller-owned.
 *
 * Synchronisation: every call is ordered on the context's CUDA stream.  Calls
 * with HOST outputs return after the results are in host memory; calls with
 * DEVICE outputs return once the work is enqueued.
 *
 * Errors: every call returns a vgicp_status; nothing throws across the ABI.
 * On error, vgicp_last_error() describes the first failure of the last call.
 * A context is used from one host thread at a time.
 */
#ifndef VGICP_H
#define VGICP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VGICP_OK = 0,
    VGICP_ERR_INVALID_ARG = 1,  /* null pointer, negative size, bad handle, r <= 0 or non-finite */
    VGICP_ERR_OOM = 2,          /* device or pinned host allocation failed */
    VGICP_ERR_NOT_FOUND = 3,    /* handle does not exist (released or never created) */
    VGICP_ERR_EMPTY = 4,        /* overlap of a source with zero points (Eq. 8 undefined) */
    VGICP_ERR_CUDA = 5,         /* a CUDA runtime call failed; see vgicp_last_error() */
    VGICP_ERR_TIMEOUT = 6,      /* a bounded device wait ran out */
    VGICP_ERR_BUDGET = 7,       /* admission would exceed the context's device-memory budget */
    VGICP_ERR_NUMERIC = 8       /* a linear system is not positive definite */
} vgicp_status;

/* Where an input or output array lives: host memory (pageable or pinned) or
 * device memory of the context's GPU.  Inputs are always copied: the kernels
 * read frames in their own padded, per-point 36 B layout (x, y, z and the six
 * covariance entries in two 16 B vectors and one float, optionally stored in
 * spatial order) with per-frame statistics and group boxes next to it, so a
 * caller's n x 3 and n x 6 arrays cannot be borrowed in place.  From device
 * memory the copy is one pass of the packing kernel (about 72 B of traffic
 * per point), enqueued on the context's current lane (see "Memory" above for
 * how long the caller's arrays must stay unchanged). */
enum { VGICP_MEM_HOST = 0, VGICP_MEM_DEVICE = 1 };

/* Linearisation precision (vgicp_options.precision). */
enum {
    /* Batched path: one persistent launch over all factors; per-point transform,
     * inverse and Jacobian products in float32.  The voxel index is exact (the
     * float32 floor on a split translation is accepted only farther than its
     * proven error bound from a voxel face, else the float64 floor is taken);
     * per-chunk sums across a warp in float32, sums of chunks in float64; 12x12
     * expansion in float64. */
    VGICP_PREC_F32 = 0,
    /* Plain path: one launch per factor; everything in float64 with the literal
     * 3x12 Jacobian and all 78 unique entries of J^T Omega J per point. */
    VGICP_PREC_F64 = 1,
    /* Batched path with a compensated transform: the point's position relative
     * to its voxel (the residual) and the lever arm come from an error-free
     * float32-pair transform instead of plain float32; the rest as
     * VGICP_PREC_F32.  Slower, about ten times more accurate residuals. */
    VGICP_PREC_F32_COMP = 2
};

typedef struct vgicp_ctx vgicp_ctx;
typedef int64_t vgicp_map_t;    /* voxelmap handle */
typedef int64_t vgicp_frame_t;  /* source-frame handle (points + covariances resident on device) */

/* One VGICP matching-cost factor (Eq. 1, 3): target voxelmap B, source frame A,
 * and the indices of T_B and T_A in the poses array passed to vgicp_linearize(). */
typedef struct {
    vgicp_map_t target;
    vgicp_frame_t source;
    int32_t target_pose;
    int32_t source_pose;
} vgicp_factor;

typedef struct {
    int32_t precision;        /* VGICP_PREC_F32 (default), VGICP_PREC_F64 or VGICP_PREC_F32_COMP */
    int32_t chunk_points;     /* points per work item of the batched path (one warp per item; multiple of 32;
                                 0 = default 2048); a factor of n points is cut into items of
                                 min(chunk_points, max(64, ceil(n / 8) rounded up to 32)) points, so that a
                                 small factor spreads over several warps (a function of n only: a factor's
                                 result is the same alone and in any batch) */
    int32_t linearize_variant;/* batched kernel variant: 0 default, 1 to 5 (same results, different
                                 latency hiding), 6 (maps of at most 4,096 voxels probed from a copy in
                                 shared memory, one CTA per SM taking runs of items with one target);
                                 chosen by measurement */
    int32_t blocks_per_sm;    /* persistent grid = SMs x this (0 = the variant's default) */
    int64_t hbm_budget_bytes; /* device bytes handles may hold in total (0 = unlimited) */
    /* 1 (default): overlap pairs whose source bounding box, moved by the pair's
     * pose and grown by a margin far above float64 rounding, misses the target's
     * voxel bounding box are answered 0 without visiting their points (exact:
     * such a pair has no correspondence), chunks of consecutive points whose
     * box misses it are skipped, and so are groups of 32 consecutive stored
     * points whose moved box reaches no occupied cell of the target's coarse
     * occupancy grid (cells of 4^3 voxels or more).  0: every point is looked up. */
    int32_t overlap_cull;
    /* 1 (default): the same exact tests per chunk and per group of 32 source
     * points (boxes kept per frame) let the linearisation skip work items and
     * groups that provably find no voxel; results are unchanged. */
    int32_t linearize_cull;
    /* Correspondences of a source point (linearisation and evaluation; the
     * overlap of Eq. 8 always uses the containing voxel): 1 (default) the voxel
     * containing the transformed point (Sec. III-A); 7 also its six face
     * neighbours; 27 every voxel of its 3x3x3 block (the DIRECT7 / DIRECT27
     * association of the earlier VGICP formulation).  Each found voxel v is a
     * correspondence of its own with e = mu_v - T_BA p; inliers count them.
     * Chunk culling is off for 7 and 27. */
    int32_t neighbors;
    /* 1: each correspondence weighted by its voxel's point count (Omega scaled
     * by it); 0 (default): unweighted, as Eq. 2, 5, 6. */
    int32_t count_weighted;
    /* Storage order of the points of frames registered from now on: 2 (default)
     * spatial within tiles -- each run of 4,096 given points sorted on its own by
     * the Morton (z-order) code of the points' cells in a 256^3 grid over the
     * frame's bounding box, ties in the given order, non-finite points last --
     * so that the lanes of a warp look up the same few voxels; a frame of any
     * size is ordered by as many blocks as it has tiles, so one frame registers
     * quickly; 1: the same order over the whole frame (one block per frame; as
     * fast for batches of hundreds of frames, slow for one large frame); 0: the
     * given order.  Results differ only by the
     * float32 summation order (overlap counts, inliers and voxelmaps are the
     * same); per-point outputs (vgicp_debug_correspondences,
     * vgicp_linearize_correspondences) are always in the given order.  A
     * spatially ordered frame holds 4 more bytes per point. */
    int32_t frame_order;
    /* 1 (default): with overlap_cull / linearize_cull, the exact tests also
     * skip groups of 32 consecutive stored points (see those options); 0: cull
     * chunks and pairs only.  Results are the same either way. */
    int32_t group_cull;
} vgicp_options;

/* Fill *opt with the defaults above. */
vgicp_status vgicp_options_default(vgicp_options *opt);

/* Create a context on the current CUDA device.  opt may be NULL (defaults).
 * cuda_stream is a cudaStream_t to order work on, or NULL for a stream the
 * context creates and owns. */
vgicp_status vgicp_create(vgicp_ctx **ctx, const vgicp_options *opt, void *cuda_stream);

/* Destroy a context: synchronises its stream and frees every handle. */
vgicp_status vgicp_destroy(vgicp_ctx *ctx);

/* Replace the options of a live context (takes effect on the next call). */
vgicp_status vgicp_set_options(vgicp_ctx *ctx, const vgicp_options *opt);

/* Order subsequent work on another stream (NULL = the context's own stream). */
vgicp_status vgicp_set_stream(vgicp_ctx *ctx, void *cuda_stream);

/* Select the lane later calls use (0 <= lane < 4).  Each lane has its own CUDA
 * stream (cuda_stream, or NULL for one the context creates on first use) and
 * its own scratch buffers, so calls on different lanes may be in flight at
 * the same time; handles and their device data are shared by all lanes.  The
 * caller must not release or rebuild a handle that another lane's enqueued
 * work still reads, and must order work that uses a handle after the work that
 * created or rebuilt it when that ran on another lane (vgicp_synchronize on
 * that lane, or a CUDA event recorded there and waited for on this lane's
 * stream): a handle's descriptor and data are written on the creating lane's
 * stream.  Lane 0 is the context's initial stream. */
vgicp_status vgicp_set_lane(vgicp_ctx *ctx, int32_t lane, void *cuda_stream);

/* Block until all work enqueued on the context's current lane has finished. */
vgicp_status vgicp_synchronize(vgicp_ctx *ctx);

/* Register a point cloud with per-point covariances as a source frame (its
 * points p_k and covariances C_k of Eq. 2).  The data are copied into a
 * coalesced device layout owned by the handle.  n may be 0. */
vgicp_status vgicp_add_frame(vgicp_ctx *ctx, const float *points, const float *covs, int64_t n,
                             int mem_kind, vgicp_frame_t *out);

/* Register m frames in one call: frame u has n[u] points, stored one frame
 * after another in points (total x 3) and covs (total x 6), total = sum n[u],
 * both in mem_kind memory; out[u] receives its handle.  The same frames as m
 * vgicp_add_frame() calls, with one copy of each array and one batched pass
 * for all of them.  All or nothing: on an error no handle is created. */
vgicp_status vgicp_add_frames(vgicp_ctx *ctx, const float *points, const float *covs, const int64_t *n, int64_t m,
                              int mem_kind, vgicp_frame_t *out);

/* Number of points of a frame. */
vgicp_status vgicp_frame_size(vgicp_ctx *ctx, vgicp_frame_t frame, int64_t *n);

/* Build the voxelmap of a cloud (in its own frame) at resolution r (Sec. III-A):
 * an open-addressing hash on the device from voxel coordinate to (point count,
 * mean, covariance).  Points with invalid voxel coordinates are skipped. */
vgicp_status vgicp_build_voxelmap(vgicp_ctx *ctx, const float *points, const float *covs, int64_t n,
                                  double resolution, int mem_kind, vgicp_map_t *out);

/* Build voxelmaps of n registered frames at resolution r in one batched pass.
 * maps[i] < 0 on input creates a new handle; maps[i] >= 0 rebuilds that map in
 * place (its device memory is reused when large enough). */
vgicp_status vgicp_build_voxelmaps(vgicp_ctx *ctx, const vgicp_frame_t *frames, int64_t n,
                                   double resolution, vgicp_map_t *maps);

/* Number of voxels of a map. */
vgicp_status vgicp_voxelmap_size(vgicp_ctx *ctx, vgicp_map_t map, int64_t *n_voxels);

/* Linearise n_f factors (Eq. 3-6) at the poses given (n_poses x 12 doubles,
 * host memory).
 * Outputs (caller-owned, n_f entries each, in out_kind memory):
 *   H  n_f x 144 doubles (full symmetric 12x12, [xi_B ; xi_A] order),
 *   b  n_f x 12 doubles, cost n_f doubles, inliers n_f int64 (nullable):
 *   the number of source points that found a target voxel.
 * Precision follows the context options (VGICP_PREC_*).  Factors whose
 * indices or handles are invalid make the whole call fail with INVALID_ARG or
 * NOT_FOUND before any work is enqueued. */
vgicp_status vgicp_linearize(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f,
                             const double *poses, int64_t n_poses,
                             double *H, double *b, double *cost, int64_t *inliers, int out_kind);

/* vgicp_linearize() with the correspondences it took recorded (Sec. III-A:
 * each transformed source point is associated with the target voxel that
 * contains it; parity checks of the linearisation's own voxel floor and hash
 * probe).  The same launch configuration, precision, variant, chunks and
 * culling as vgicp_linearize(); the kernels are the recording instantiations
 * of the same code, so H, b, cost and inliers equal vgicp_linearize()'s.
 * Point j of factor f's source is entry e = (sum of the source sizes of
 * factors 0..f-1) + j of:
 *   keys   3 int64 per entry: the voxel coordinate the kernel computed for the
 *          point under T_target_source, INT64_MIN on every axis when it has
 *          none (a coordinate outside [-2^20, 2^20 - 1] or not finite) or was
 *          never visited;
 *   state  int32 per entry: 1 when that voxel exists in the target map, 0 when
 *          not, -1 when the point lies in a chunk the exact culling skipped
 *          (provably no voxel); with neighbour association (options.neighbors
 *          7 or 27), bit o set when the voxel at neighbour offset o exists.
 * keys and state are host arrays sized for the sum of the factors' source
 * sizes (required); H, b, cost, inliers are host arrays as for
 * vgicp_linearize() and may all be NULL.  Errors as vgicp_linearize(). */
vgicp_status vgicp_linearize_correspondences(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f,
                                             const double *poses, int64_t n_poses,
                                             double *H, double *b, double *cost, int64_t *inliers,
                                             int64_t *keys, int32_t *state);

/* Error evaluation (Sec. III-D: the optimiser evaluates the summed matching
 * cost of Eq. 1 to accept or reject a step): each factor's cost
 * sum e' Omega e and inlier count at the given poses, by the batched path with
 * only the cost accumulated -- the same chunks, order and kernel variant as
 * vgicp_linearize(), so the costs agree with its cost output bit for bit.
 * Runs VGICP_PREC_F32 (or VGICP_PREC_F32_COMP when set; VGICP_PREC_F64 runs as
 * VGICP_PREC_F32).  cost and inliers (nullable): n_f entries in out_kind memory. */
vgicp_status vgicp_evaluate(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f, const double *poses,
                            int64_t n_poses, double *cost, int64_t *inliers, int out_kind);

/* Autotuner for the batched float32 linearisation (Sec. III-D's "issue all
 * factors, then synchronise" step): times every candidate (kernel variant x
 * points per work item x persistent grid) on this factor set with CUDA events
 * on the context stream, `reps` timed runs each after one warm-up, and keeps
 * the fastest in the context options (VGICP_PREC_F64 becomes VGICP_PREC_F32;
 * VGICP_PREC_F32_COMP is kept).
 * best (nullable) receives those options and best_ms (nullable) the time of one
 * run.  Results differ between candidates only by float32 summation order. */
vgicp_status vgicp_autotune(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f, const double *poses,
                            int64_t n_poses, int32_t reps, vgicp_options *best, double *best_ms);

/* Gauss-Newton iteration plan.  The global optimisation of Sec. III-D
 * re-linearises the same factor set at new poses every iteration; a plan
 * fixes that set once and runs each iteration as one CUDA graph (pose upload,
 * per-factor pose preparation, the persistent batched float32 linearisation,
 * the fixed-order per-factor reduction), so an iteration costs one graph
 * launch instead of per-call validation, work-list and launch overhead.
 * Results are bit-identical to vgicp_linearize() with the same options.
 *
 * The plan keeps the factor handles and reads their device data at run time,
 * so voxelmaps rebuilt in place between iterations are used as they are then.
 * A plan run after a handle was released returns VGICP_ERR_NOT_FOUND; one run
 * after the options (chunk_points, variant, blocks_per_sm, linearize_cull) or
 * the context's descriptor tables changed captures its graph again first.
 * Plans are destroyed before their context; a plan is used by one host thread
 * at a time and runs on the context's current lane. */
typedef struct vgicp_plan vgicp_plan;

/* Fix n_f factors whose pose indices are < n_poses, capture the graph. */
vgicp_status vgicp_plan_create(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f, int64_t n_poses,
                               vgicp_plan **plan);

/* One iteration: poses n_poses x 12 doubles (host, copied into the plan's
 * pinned staging buffer before the call returns; a run first waits until the
 * previous run of this plan has read it).  H, b, cost, inliers (nullable) as
 * for vgicp_linearize(), in out_kind memory; HOST outputs return synchronised,
 * DEVICE outputs are written in stream order.  Needs VGICP_PREC_F32 or
 * VGICP_PREC_F32_COMP. */
vgicp_status vgicp_plan_linearize(vgicp_ctx *ctx, vgicp_plan *plan, const double *poses, double *H, double *b,
                                  double *cost, int64_t *inliers, int out_kind);

/* Number of runs and of graph captures so far (either may be NULL). */
vgicp_status vgicp_plan_info(vgicp_ctx *ctx, const vgicp_plan *plan, int64_t *runs, int64_t *captures);

/* Wait for the plan's last run and free it. */
vgicp_status vgicp_plan_destroy(vgicp_ctx *ctx, vgicp_plan *plan);

/* Size limits of vgicp_linearize_noalloc() (its fixed scratch is sized for them). */
#define VGICP_NOALLOC_MAX_FACTORS 1024
#define VGICP_NOALLOC_MAX_POSES 2048
#define VGICP_NOALLOC_MAX_ITEMS 16384   /* sum over factors of their work items (see chunk_points) */

/* vgicp_linearize() without any allocation.  The paper has no counterpart:
 * this serves callers that must not allocate device memory when they
 * linearise, for example a mapping loop that fixes its device-memory footprint
 * at start-up so an optimiser iteration cannot fail for lack of memory, or an
 * application whose own allocator owns all device memory.  They create the
 * context, frames and voxelmaps beforehand and pass their own outputs.
 *
 * Results equal vgicp_linearize()'s bit for bit with the context's batched
 * precision (VGICP_PREC_F32, or VGICP_PREC_F32_COMP when set; VGICP_PREC_F64
 * runs as VGICP_PREC_F32), chunk_points and linearize_variant: each factor is
 * cut into the same chunks, each chunk's sums are taken by one warp in the same
 * point and lane order, and each factor's chunk sums are added in chunk order
 * (only the order in which chunks are listed differs).  Variant 6 (the
 * shared-memory map path) runs as the default variant, whose per-chunk
 * arithmetic and lane order are the same.
 * factors and poses are host arrays copied on the context stream (a pinned
 * buffer must stay valid until the stream passes the copy); H (n_f x 144),
 * b (n_f x 12), cost (n_f) and inliers (n_f, nullable) are DEVICE memory,
 * written asynchronously.  Sizes beyond VGICP_NOALLOC_MAX_FACTORS,
 * VGICP_NOALLOC_MAX_POSES or VGICP_NOALLOC_MAX_ITEMS return
 * VGICP_ERR_INVALID_ARG; unknown handles VGICP_ERR_NOT_FOUND.
 *
 * All intermediate data lives in one fixed device array of about 4.5 MB that
 * every GPU loading the library holds until the process exits.  The first call
 * on a device looks up that array's device address (the device must be
 * current); make that first call before any stream capture.  Every call
 * reuses the array: calls whose work overlaps on the GPU race on it. */
vgicp_status vgicp_linearize_noalloc(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f,
                                     const double *poses, int64_t n_poses,
                                     double *H, double *b, double *cost, int64_t *inliers);

/* Overlap of a source frame with a target voxelmap (Eq. 8) under the relative
 * pose T_target_source (12 doubles, host): fraction = count / N.  count is
 * optional (nullable).  N = 0 returns VGICP_ERR_EMPTY. */
vgicp_status vgicp_overlap(vgicp_ctx *ctx, vgicp_frame_t source, vgicp_map_t target,
                           const double *T_target_source, double *fraction, int64_t *count);

/* Overlap counts of n listed pairs (Eq. 7-8 numerators): counts[i] = #{k :
 * voxel(T_i p_k) in targets[i]} for the points p_k of sources[i], T n x 12
 * doubles (host, target-from-source).  counts int64 in out_kind memory.
 * Sources with N = 0 give count 0 (the caller decides what Eq. 8 means then). */
vgicp_status vgicp_overlap_pairs(vgicp_ctx *ctx, const vgicp_frame_t *sources, const vgicp_map_t *targets,
                                 int64_t n, const double *T, int64_t *counts, int out_kind);

/* Overlap counts of every (source, target) pair (Eq. 7-8 numerators):
 * counts[s * n_tgt + t] = #{k : voxel(T_t^-1 T_s p_k) in map t}, poses_src
 * n_src x 12 and poses_tgt n_tgt x 12 (world-from-frame, host).  counts is
 * caller-owned int64 in out_kind memory. */
vgicp_status vgicp_overlap_matrix(vgicp_ctx *ctx, const vgicp_frame_t *sources, int64_t n_src,
                                  const vgicp_map_t *targets, int64_t n_tgt,
                                  const double *poses_src, const double *poses_tgt,
                                  int64_t *counts, int out_kind);

/* Work of the last vgicp_overlap_matrix() call on this context: the number of
 * pairs not culled and the number of point lookups performed (the points of
 * the groups of 32 stored points that the exact culling could not rule out).
 * Synchronises the context stream. */
vgicp_status vgicp_overlap_matrix_work(vgicp_ctx *ctx, int64_t *live_pairs, int64_t *lookups);

/* Per-point voxel association of a source against a target (debug / parity):
 * keys (n x 3 int64, host) receives each point's voxel coordinate under
 * T_target_source (INT64_MIN on every axis when invalid), hit (n int32, host)
 * 1 if that voxel exists in the map.  Either output may be NULL. */
vgicp_status vgicp_debug_correspondences(vgicp_ctx *ctx, vgicp_frame_t source, vgicp_map_t target,
                                         const double *T_target_source, int64_t *keys, int32_t *hit);

/* Copy a voxelmap to host, sorted by (kx, ky, kz).  *n_voxels is the capacity of
 * the outputs on input and the number of voxels on output (outputs may all be
 * NULL to query the size).  keys V x 3 int64, counts V int64, mu V x 3 doubles
 * (absolute coordinates), cov V x 6 doubles. */
vgicp_status vgicp_export_voxelmap(vgicp_ctx *ctx, vgicp_map_t map, int64_t *keys, int64_t *counts,
                                   double *mu, double *cov, int64_t *n_voxels);

/* Per-point covariances from the k nearest neighbours of each point (Sec. III:
 * estimated from k neighbouring points; the point itself counts, ties go to the
 * lower index), regularised to eigenvalues (1, 1, eps): the direction of least
 * spread receives eps.  points n x 3 and covs_out n x 6 float32, both in
 * mem_kind memory.  1 <= k <= 32.  Points with fewer than k finite neighbours
 * get the identity. */
vgicp_status vgicp_estimate_covariances(vgicp_ctx *ctx, const float *points, int64_t n, int32_t k,
                                        double eps, float *covs_out, int mem_kind);

/* Release a map or frame handle and its device memory. */
vgicp_status vgicp_release(vgicp_ctx *ctx, int64_t handle);

/* Release n handles (all are checked first: an unknown handle releases none;
 * a handle listed twice fails when it is reached the second time). */
vgicp_status vgicp_release_many(vgicp_ctx *ctx, const int64_t *handles, int64_t n);

/* Device bytes a handle holds: a frame of n points (is_map = 0) or a voxelmap
 * built from n points (is_map = 1; building it also needs the n-point frame
 * it is built from).  For admission control under hbm_budget_bytes. */
vgicp_status vgicp_memory_estimate(vgicp_ctx *ctx, int64_t n, int32_t is_map, int64_t *bytes);

/* Device bytes currently held by handles of this context. */
vgicp_status vgicp_memory_in_use(vgicp_ctx *ctx, int64_t *bytes);

/* Number of kernels this context has launched since creation. */
vgicp_status vgicp_kernel_launches(vgicp_ctx *ctx, int64_t *count);

/* Device time of the hot kernels, from CUDA events recorded on the launching
 * lane's stream around each launch: vgicp_linearize's batched kernel (with the
 * reset of its work counter), vgicp_overlap_matrix's matrix kernel, and
 * vgicp_build_voxelmap(s)'s build kernels as one span.  Launches inside a
 * plan's CUDA graph are not timed.  vgicp_kernel_timing waits for the recorded
 * launches of `kernel` on the current lane since the last reset (at most 1,024)
 * and returns their summed milliseconds and their number;
 * vgicp_kernel_timing_reset forgets the current lane's records. */
enum { VGICP_KERNEL_LINEARIZE = 0, VGICP_KERNEL_OVERLAP_MATRIX = 1, VGICP_KERNEL_VOXELMAP_BUILD = 2 };
vgicp_status vgicp_kernel_timing(vgicp_ctx *ctx, int32_t kernel, double *total_ms, int64_t *launches);
vgicp_status vgicp_kernel_timing_reset(vgicp_ctx *ctx);

/* Text of the last error of this context ("" if none).  Valid until the next call. */
const char *vgicp_last_error(const vgicp_ctx *ctx);

/* ------------------------------------------------------------------------
 * Gauss-Newton / Levenberg-Marquardt (Sec. III-D: every factor is linearised
 * on the GPU, the linear system is collected and solved on the host).  The
 * factor blocks H_f, b_f of vgicp_linearize() define the Gauss-Newton model of
 * the summed cost F = sum cost_f around the current poses,
 *     F(d) = F + 2 b' d + d' H d,   d = (omega, v) per pose, T <- T Exp(d),
 * with H and b assembled from the factors' [xi_B ; xi_A] blocks.
 * ---------------------------------------------------------------------- */

/* Host only (no device work): the damped step (H + lambda D) d = -b with the
 * anchor pose held fixed (d = 0 there), D = diag(H) floored at 1e-12 of its
 * mean (plus that floor), solved by a sparse Cholesky factorisation (reverse
 * Cuthill-McKee pose order, envelope storage).  pairs: n_f x 2 int32
 * (target_pose, source_pose); H n_f x 144, b n_f x 12 as vgicp_linearize()
 * writes them; delta: n_poses x 6 out.  model_decrease (nullable) receives
 * F(0) - F(d) of the undamped model.  VGICP_ERR_NUMERIC if the damped system
 * is not positive definite.  The factorisation uses AVX2/FMA where the host has
 * them (VGICP_HOST_SIMD=0 in the environment selects portable loops; the two
 * agree to rounding). */
vgicp_status vgicp_solve_step(const int32_t *pairs, const double *H, const double *b, int64_t n_f, int64_t n_poses,
                              int32_t anchor, double lambda, double *delta, double *model_decrease);

/* Host only: T_p <- T_p Exp(delta_p) for every pose (12 doubles each, in place),
 * Exp the SE(3) exponential of (omega, v). */
vgicp_status vgicp_se3_retract(double *poses, const double *delta, int64_t n_poses);

typedef struct {
    int32_t max_iterations;     /* 0 = 20 */
    int32_t anchor;             /* pose held fixed (the gauge) */
    double lambda_init;         /* initial damping, 0 = 1e-4 */
    double relative_tolerance;  /* stop once an accepted step lowers F by less than this fraction (0 = 1e-6) */
} vgicp_lm_options;

typedef struct {
    int32_t iterations, accepted, n_history;
    int32_t reserved;
    double initial_cost, final_cost, lambda;
    double linearize_ms, evaluate_ms, solve_ms;   /* host wall time per phase */
    double history[64];                           /* F at the start and after each accepted step */
} vgicp_lm_report;

/* Levenberg-Marquardt over the factors: poses (n_poses x 12, host) are updated
 * in place.  Each iteration linearises through a plan (one CUDA graph), solves
 * vgicp_solve_step on the host, evaluates the trial poses with
 * vgicp_evaluate(), and accepts (damping / 10) or rejects (damping x 10) the
 * step.  It stops after max_iterations, when an accepted step lowers F by less
 * than relative_tolerance F, or when the Gauss-Newton model predicts less than
 * that.  Correspondences are re-associated at every linearisation. */
vgicp_status vgicp_optimize(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f, double *poses,
                            int64_t n_poses, const vgicp_lm_options *opt, vgicp_lm_report *report);

/* SE(3) loop constraint (Sec. III-D, Eq. 10-11): an explicit relative pose
 * measurement T_ij ~ T_i^-1 T_j with residual r = Log(T_ij^-1 T_i^-1 T_j)
 * (twist (omega, v)), constant information Omega (6x6, row-major), and the
 * shifted Tukey kernel on the whitened error norm x = sqrt(r' Omega r): weight
 * psi(x) = (max(0, 1 - (x - offset)^2 / width))^2.  The factor's cost is the loss
 * rho(x^2) = int_0^x psi(u) 2u du (so d rho / d(x^2) = psi), and its Gauss-Newton
 * blocks are psi(x) J' Omega J and psi(x) J' Omega r with psi frozen at the
 * linearisation point. */
typedef struct {
    int32_t pose_i, pose_j;
    double T_ij[12];
    double information[36];
    double width;
    double offset;
} vgicp_loop_factor;

/* Host only: cost (n_loops), and when non-NULL the blocks H (n_loops x 144, order
 * [xi_i ; xi_j]) and b (n_loops x 12) of the loop factors at the poses. */
vgicp_status vgicp_loop_linearize(const vgicp_loop_factor *loops, int64_t n_loops, const double *poses,
                                  int64_t n_poses, double *H, double *b, double *cost);

/* vgicp_optimize() with SE(3) loop factors added to the matching cost factors:
 * F = sum of the factors' costs + sum of the loop factors' losses. */
vgicp_status vgicp_optimize_with_loops(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f,
                                       const vgicp_loop_factor *loops, int64_t n_loops, double *poses,
                                       int64_t n_poses, const vgicp_lm_options *opt, vgicp_lm_report *report);

/* Human-readable name of a status code. */
const char *vgicp_status_string(vgicp_status s);

/* ------------------------------------------------------------------------
 * Serving loop.  An online mapper (Sec. IV's online mapping and loop closing)
 * keeps adding frames and asks, at uneven rates and sizes, for overlaps
 * (Eq. 8) to pick factor candidates and for linearisations (Eq. 3-6) of the
 * factors it keeps.  A server owns one context and one scheduler thread that
 * runs the requests submitted by any number of client threads in continuous
 * batches: whenever one of its lanes is free it launches every pending
 * request that fits (one batched linearisation plus one batched overlap
 * list), so batches overlap on the device.  Target clouds and source frames
 * are registered once under caller keys; the server keeps host copies and
 * makes them resident on demand (targets as voxelmaps), releasing the least
 * recently used idle ones when the device-memory budget would be exceeded.
 * Admission works on up to 64 pending requests at a time: as many of them,
 * from the front, as the budget can hold have their missing objects made
 * resident together (one registration of all their frames, one voxelmap build
 * per resolution); the rest wait in arrival order.  A request's result is bit-identical to the same request run alone: the
 * batched float32 linearisation sums fixed chunks in a fixed order and
 * overlap counts are exact.
 * ---------------------------------------------------------------------- */
typedef struct vgicp_server vgicp_server;

typedef struct {
    int64_t hbm_budget_bytes;    /* device bytes resident maps and frames may hold (0 = unlimited) */
    int32_t max_batch_requests;  /* requests per batch (0 = 4096) */
    int32_t lanes;               /* concurrent batches, 1..4 (0 = 2) */
    int64_t max_batch_points;    /* source points per batch (0 = 2^27); a larger single request still runs */
    int32_t device_loop;         /* 1: device-resident request loop (below) instead of host-launched batches */
    int32_t loop_slots;          /* device loop: requests in flight at most (0 = 256, at most 1024) */
    double loop_idle_ms;         /* device loop: the loop kernel ends after this long without a request
                                    (0 = 20 ms); the next request starts it again */
} vgicp_server_options;

enum { VGICP_REQ_LINEARIZE = 0, VGICP_REQ_OVERLAP = 1 };

typedef struct {
    int32_t kind;                /* VGICP_REQ_LINEARIZE or VGICP_REQ_OVERLAP */
    int32_t reserved;            /* 0 */
    int64_t target;              /* key given to vgicp_server_put_map() */
    int64_t source;              /* key given to vgicp_server_put_frame() */
    double T_target_source[12];  /* relative pose T_BA, row-major 3x4, finite */
} vgicp_request;

typedef struct {
    vgicp_status status;         /* VGICP_OK, or why the request failed (VGICP_ERR_BUDGET: the pair
                                    cannot fit the budget even with everything else released) */
    int32_t kind;
    double H[144];               /* LINEARIZE: as vgicp_linearize() with T_target = I, T_source = T_BA */
    double b[12];
    double cost;
    int64_t count;               /* LINEARIZE: inliers; OVERLAP: points with a target voxel */
    double fraction;             /* OVERLAP: count / N (status VGICP_ERR_EMPTY when N = 0) */
    double latency_ms;           /* submit to completion, host clock */
} vgicp_result;

typedef struct {
    int64_t submitted, completed, batches, admissions, evictions;
    int64_t resident_bytes;      /* device bytes held by resident maps and frames */
    double mean_batch_requests;
    double p50_ms, p99_ms, max_ms; /* latency quantiles of completed requests */
    double host_launch_ms;       /* scheduler time spent admitting and launching batches */
    double host_finish_ms;       /* scheduler time spent handing results out */
    double device_ms;            /* device time of the batches (event-timed on each lane's stream) */
    double host_admit_ms;        /* part of host_launch_ms spent making objects resident */
    double host_enqueue_ms;      /* part of host_launch_ms spent in the batched library calls */
} vgicp_server_counters;

/* Create a server on the current CUDA device.  opt and kernel_opt (kernel
 * variant, chunk size, culling; precision is forced to VGICP_PREC_F32) may be
 * NULL for defaults. */
vgicp_status vgicp_server_create(vgicp_server **server, const vgicp_server_options *opt,
                                 const vgicp_options *kernel_opt);

/* Finish every batch in flight, stop the scheduler and free everything.
 * Requests still pending are dropped. */
vgicp_status vgicp_server_destroy(vgicp_server *server);

/* Register a target cloud (n x 3 points, n x 6 covariances, host float32) to be
 * voxelised at resolution r.  The data are copied.  Keys are 0 <= key < 2^62;
 * a key already registered returns VGICP_ERR_INVALID_ARG. */
vgicp_status vgicp_server_put_map(vgicp_server *server, int64_t key, const float *points, const float *covs,
                                  int64_t n, double resolution);

/* Register a source frame (host float32, copied).  Same key rules; maps and
 * frames have separate key spaces. */
vgicp_status vgicp_server_put_frame(vgicp_server *server, int64_t key, const float *points, const float *covs,
                                    int64_t n);

/* Queue a request; *ticket identifies it to vgicp_server_wait().  Unknown keys
 * return VGICP_ERR_NOT_FOUND and queue nothing.  Thread-safe. */
vgicp_status vgicp_server_submit(vgicp_server *server, const vgicp_request *req, int64_t *ticket);

/* Queue n requests at once (all or none: any invalid request or unknown key
 * fails the call before anything is queued); tickets[k] for reqs[k]. */
vgicp_status vgicp_server_submit_batch(vgicp_server *server, const vgicp_request *reqs, int64_t n, int64_t *tickets);

/* Wait up to timeout_s seconds (< 0: no limit) for a request; on VGICP_OK *out
 * holds its result (whose own status may be an error) and the ticket is
 * retired.  VGICP_ERR_TIMEOUT leaves the ticket valid.  Thread-safe. */
vgicp_status vgicp_server_wait(vgicp_server *server, int64_t ticket, double timeout_s, vgicp_result *out);

/* vgicp_server_wait() for n tickets in order, results to out[0..n).  On
 * VGICP_ERR_TIMEOUT the tickets already returned are retired, the rest stay
 * valid; an unknown ticket fails the call before anything is retired. */
vgicp_status vgicp_server_wait_batch(vgicp_server *server, const int64_t *tickets, int64_t n, double timeout_s,
                                     vgicp_result *out);

/* Counters and latency quantiles since creation or the last reset. */
vgicp_status vgicp_server_stats(vgicp_server *server, vgicp_server_counters *out);
vgicp_status vgicp_server_reset_stats(vgicp_server *server);

/* Text of the server's last error ("" if none). */
const char *vgicp_server_last_error(const vgicp_server *server);

/* Device-resident request loop (options.device_loop = 1; Sec. III-D issues each
 * factor's evaluation to the GPU on its own, Sec. IV's online mapper issues
 * them as frames arrive).  Requests are not batched on the host: each admitted
 * request is written into a ring of slots in page-locked host memory that the
 * device reads directly, and one persistent kernel picks it up while earlier
 * requests are still running -- a dispatcher warp splits it into chunks on a
 * device work queue, every other warp of the grid takes chunks as they come,
 * and the warp finishing a request's last chunk writes the result straight
 * into the ring's result slot, which the server hands to the waiter.  A
 * request's chunks, their per-chunk sums and the chunk-order reduction are
 * those of vgicp_linearize(), so a result equals vgicp_linearize() of that
 * factor (T_target = I, T_source = T_BA, same kernel options) bit for bit,
 * alone or amid other requests; overlap counts are exact.  Residency, the
 * budget and LRU eviction work as in batch mode; a request pins its map and
 * frame until its result is read.  Every wait in the kernel is bounded: when
 * no request arrives for loop_idle_ms the loop kernel ends with
 * VGICP_ERR_TIMEOUT (not an error of any request) and the next request
 * launches it again.  Requests need at most 128 chunks of the context's
 * chunk_points (262,144 source points at the default); larger ones complete
 * with VGICP_ERR_INVALID_ARG.  Needs the single-voxel, unweighted association
 * (kernel_opt.neighbors <= 1, count_weighted 0).
 *
 * State of the loop kernel: *running 1 while it runs, *last_exit the status
 * it ended with last time (VGICP_OK before the first end; VGICP_ERR_TIMEOUT
 * after an idle end), *launches how often it was started (any may be NULL).
 * VGICP_ERR_INVALID_ARG for a server without the device loop. */
vgicp_status vgicp_server_loop_state(vgicp_server *server, int32_t *running, int32_t *last_exit,
                                     int64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* VGICP_H */
