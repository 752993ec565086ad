// Host-side launchers of the VGICP kernels (declarations shared by the .cu files).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "vgicp_internal.cuh"

namespace vg {

// A work item: `count` consecutive points of one unit (a map being built, a
// factor, or an overlap pair) starting at point `start` of that unit's frame.
struct __align__(16) WorkItem {
    int32_t unit;
    int32_t count;
    int64_t start;
};

// ----------------------------------------------------------- frames ------
// Re-lay n points (n x 3) and covariances (n x 6) into the three frame streams
// and gather the frame statistics (stats initialised as the kStat* layout says).
void launch_frame_pack(const float *points, const float *covs, int64_t n, float4 *pa, float4 *pb, float *pc,
                       float *stats, cudaStream_t st);

// Register m frames from staged points / covariances (frame u's at src_off[u]):
// descriptors into the table, statistics, the streams and the cull-chunk
// bounding boxes (2^shift points each).  Frames whose descriptor has a perm
// array are stored in spatial order (order_scratch: 4 x total uint32, required
// when order_mode is 1).  order_mode: 0 the given order; 1 spatial order of
// each whole frame; 2 spatial order within each 4,096-point registration item
// (points stay in their tile; no scratch).  Every frame then has a perm array.
void launch_frames_register(const float *pts, const float *cov, const int64_t *src_off, const int32_t *fidx, int m,
                            const WorkItem *items, int n_items, const WorkItem *chunks, int n_chunks,
                            const uint32_t *desc_idx, const FrameDesc *descs, FrameDesc *table, uint32_t *order_scratch,
                            int64_t total, int num_sms, int order_mode, cudaStream_t st);
void launch_chunk_boxes(const float4 *pa, int64_t n, int shift, int nchunks, float *cbox, cudaStream_t st);

// Write n map descriptors into the device table: table[idx[i]] = src[i].
void launch_scatter_map_descs(const uint32_t *idx, const MapDesc *src, int n, MapDesc *table, cudaStream_t st);

// ----------------------------------------------------------- voxelmaps ---
// Scratch of a batched build: per point the slot it went to; per voxel the
// exact fixed-point sums; per map the voxel counter.
struct BuildScratch {
    int32_t *slot_of_point;   // total points
    int64_t *acc;             // 10 x total points (worst case: every point its own voxel)
    int32_t *vid_of_slot;     // total capacity
    int32_t *slot_of_vid;     // total points
};

struct BuildUnit {
    int32_t map;         // index into the MapDesc table
    int32_t frame;       // index into the FrameDesc table
    int64_t point_base;  // offset of this unit's points in the scratch arrays
    int64_t slot_base;   // offset of this unit's slots in vid_of_slot
    uint32_t *n_voxels;  // the map's voxel counter (in the map's own allocation)
    int64_t pad;
};

void launch_voxelmap_build(const MapDesc *maps, const FrameDesc *frames, const BuildUnit *units, int n_units,
                           const WorkItem *items, int n_items, BuildScratch scr, int grid, cudaStream_t st);
// Shared-memory images of the maps idx[0..n) (table indices), made on demand.
void launch_map_images(const MapDesc *maps, const int32_t *idx, int n, int num_sms, cudaStream_t st);

// ----------------------------------------------------------- linearise ---
// Relative poses T_BA = T_B^-1 T_A for every factor, in the forms the kernels use.
void launch_prepare_factors(const int32_t *factor_idx /* n_f x 4: map, frame, pose_t, pose_s */, int n_f,
                            const double *poses, const MapDesc *maps, const FrameDesc *frames, int cull,
                            PoseParam *out, cudaStream_t st);

// n pairs with given relative poses T (n x 12 doubles, device).
void launch_prepare_list(const double *T, const int32_t *map_idx, const int32_t *frame_idx, int n,
                         const MapDesc *maps, const FrameDesc *frames, int cull, PoseParam *out, cudaStream_t st);

// One pair with a given relative pose T (12 doubles, device).
void launch_prepare_given(const double *T, int map, int frame, const MapDesc *maps, const FrameDesc *frames,
                          int cull, PoseParam *out, cudaStream_t st);

// Per-point record of the correspondences one linearisation pass took (parity
// checks of the hot path's own floor and probe).  For point i of factor f's
// source, at j = base[f] + i: key[j] = the packed voxel coordinate the kernel
// computed for the point (kEmptyKey when it has none: out of range, not
// finite), state[j] = 1 when that voxel was found in the target map, 0 when not
// (with neighbour association: bit o set when the voxel at neighbour offset o
// was found).  Points the kernel never visits (culled chunks) keep whatever the
// caller stored there.  A null key pointer turns recording off.
struct CorrRecord {
    uint64_t *key;
    int32_t *state;
    const int64_t *base;
};

// Batched float32 path: one persistent launch over all work items (one warp per
// item at a time); each item writes 28 float64 partial sums and an inlier
// count.  variant: 0 default, 1 and 2 alternatives (see linearize.cu);
// grid_per_sm: blocks per SM of the persistent grid (0 = the variant's own).
// rec: when rec.key is set, a recording instantiation of the same kernel also
// writes every visited point's correspondence.
void launch_linearize_f32(const PoseParam *params, const MapDesc *maps, const FrameDesc *frames,
                          const WorkItem *items, int n_items, double *partials, int64_t *inl_partials,
                          int *next_item, int variant, int grid_per_sm, int num_sms, bool compensated, int nb,
                          int weighted, cudaStream_t st, CorrRecord rec = CorrRecord{});

// Per-factor fixed-order float64 reduction of the item partials and expansion
// to the 12x12 H, b, cost.  item_begin has n_f + 1 entries.
void launch_linearize_img(const PoseParam *params, const MapDesc *maps, const FrameDesc *frames,
                          const WorkItem *items, const int4 *units, int n_units, double *partials,
                          int64_t *inl_partials, int *next_unit, int num_sms, bool compensated, cudaStream_t st,
                          CorrRecord rec = CorrRecord{});
void launch_cost_f32(const PoseParam *params, const MapDesc *maps, const FrameDesc *frames, const WorkItem *items,
                     int n_items, double *partials, int64_t *inl_partials, int *next_item, int variant,
                     int grid_per_sm, int num_sms, bool compensated, int nb, int weighted, cudaStream_t st);
void launch_reduce_cost(const int32_t *item_range, int n_f, const double *partials, const int64_t *inl_partials,
                        double *cost, int64_t *inliers, cudaStream_t st);
void launch_reduce_finalize(const PoseParam *params, const int32_t *item_range, int n_f, const double *partials,
                            const int64_t *inl_partials, double *H, double *b, double *cost, int64_t *inliers,
                            cudaStream_t st);

// Plain float64 path for one factor (literal Jacobians, 78 unique H entries).
// scratch holds grid x 92 doubles; ticket is one zeroed int (reset by the kernel).
// rec_key / rec_state (nullable): this factor's per-point record (CorrRecord
// layout, already offset to the factor's first point).
void launch_linearize_f64(const PoseParam *param, const MapDesc *maps, const FrameDesc *frames, int64_t n,
                          double *scratch, unsigned int *ticket, double *H, double *b, double *cost,
                          int64_t *inliers, int grid, int nb, int weighted, cudaStream_t st,
                          uint64_t *rec_key = nullptr, int32_t *rec_state = nullptr);
int linearize_f64_block();

// ----------------------------------------------------------- overlap -----
// counts[unit] += #hits of the unit's points (counts must be zeroed).
void launch_overlap(const PoseParam *params, const MapDesc *maps, const FrameDesc *frames, const WorkItem *items,
                    int n_items, unsigned long long *counts, int grid, cudaStream_t st);

// Overlap matrix: counts[s * n_tgt + t] += hits of source s against target t
// (pairs[s * n_tgt + t] prepared by launch_prepare_pairs).  Items whose target
// table fits 64 KB run on two 512-thread CTAs per SM, the others on one
// 1024-thread CTA per SM.
size_t overlap_matrix_scratch_bytes(int n_src, int n_tgt);
void launch_overlap_matrix(const PoseParam *pairs, const MapDesc *maps, const FrameDesc *frames, int n_src,
                           int n_tgt, unsigned long long *counts, void *scratch, int num_sms,
                           cudaStream_t st);

// out[0] += pairs not culled, out[1] += the points the matrix kernel visits for
// them (points of live groups in live cull chunks) (out zeroed).
void launch_count_live(const PoseParam *pairs, int64_t n_pairs, const FrameDesc *frames, const MapDesc *maps,
                       unsigned long long *out, cudaStream_t st);

// Pair parameters of an overlap matrix: pair (s, t) -> T_t^-1 T_s; with cull set,
// pairs whose source bounding box cannot meet the target's voxels are flagged.
void launch_prepare_pairs(const double *poses_src, const double *poses_tgt, const int32_t *frame_idx,
                          const int32_t *map_idx, int n_src, int n_tgt, const MapDesc *maps,
                          const FrameDesc *frames, int cull, PoseParam *out, cudaStream_t st);

// Per-point association (debug / parity): keys n x 3 (INT64_MIN if invalid), hit n.
void launch_correspondences(const PoseParam *param, const MapDesc *maps, const FrameDesc *frames, int64_t n,
                            int64_t *keys, int32_t *hit, cudaStream_t st);

// Export: gather the occupied slots of a map (compacted, unordered).
void launch_export_voxels(const MapDesc *map_dev, uint32_t cap, uint32_t *counter, uint64_t *keys_out,
                          VoxelRec *rec_out, cudaStream_t st);

// ----------------------------------------------------------- covariances --
// kNN covariances on a uniform grid of cell size h (any h gives the same result).
size_t knn_scratch_bytes(int64_t n);
void launch_knn_covariances(const float *points, int64_t n, int k, double eps, double h, void *scratch, float *covs,
                            cudaStream_t st);

}  // namespace vg

// --------------------------------------------------- context access -------
struct vgicp_ctx;


namespace vg {

struct CtxView {
    cudaStream_t stream;
    int device, num_sms, chunk, variant, blocks_per_sm, linearize_cull;
    bool compensated;
    int neighbors, count_weighted;
    MapDesc *d_maps;
    FrameDesc *d_frames;
};

bool ctx_view(::vgicp_ctx *ctx, CtxView *v);
bool ctx_is_map(::vgicp_ctx *ctx, int64_t handle);
bool ctx_frame_size(::vgicp_ctx *ctx, int64_t handle, int64_t *n);
void ctx_count_launches(::vgicp_ctx *ctx, int n);
// Descriptors of a resident map and frame (copies of the host mirrors) and the
// frame's point count; false for an unknown handle.
bool ctx_descs(::vgicp_ctx *ctx, int64_t map, int64_t frame, MapDesc *m, FrameDesc *f, int64_t *n_points);
// vgicp_add_frames for m frames whose host arrays lie apart: frame u's points
// (n[u] x 3) and covariances (n[u] x 6) at points[u] and covs[u], each copied
// into the current lane's staging buffer, then registered in one batched pass.
// Returns a vgicp_status.
int ctx_add_frames_gather(::vgicp_ctx *ctx, const float *const *points, const float *const *covs, const int64_t *n,
                          int64_t m, int64_t *out);

}  // namespace vg

namespace vg {

// ------------------------------------------------ device request loop ----
// A persistent kernel serving linearisation and overlap requests that the
// host publishes, one at a time, into a ring of slots in page-locked host
// memory mapped into the device's address space.  Request r lives in slot
// r % slots; the host writes its fields, then its seq (= r + 1) with release
// order.  One dispatcher warp waits for the next request, prepares its pose
// parameters and appends its chunks to a device work queue; every other warp
// takes chunks from the queue, computes them as the batched kernels do, and
// the warp that finishes a request's last chunk adds the chunk sums in chunk
// order into the request's result slot, then writes the result's done word
// (= seq) with release order at system scope.  Every wait is bounded: the
// dispatcher gives up when no request arrives for idle_ns (the loop then ends
// with VGICP_ERR_TIMEOUT in LoopExit), a worker when the dispatcher has
// signalled the end and no chunk is left, or after worker_ns without either.
// The host can also end the loop through LoopExit::stop.
constexpr int kLoopMaxItems = 128;      // chunks per request
constexpr int kLoopBlock = 256;
enum { kLoopLinearize = 0, kLoopOverlap = 1 };

struct __align__(16) LoopRequest {      // host -> device, one per slot
    MapDesc map;
    FrameDesc frame;
    double T[12];                       // T_target_source (T_BA)
    int32_t kind;                       // kLoopLinearize or kLoopOverlap
    int32_t n_items;                    // chunks (1 .. kLoopMaxItems)
    int32_t chunk;                      // points per chunk (the last takes the rest)
    int32_t cull;                       // exact culling: 0 none, 1 chunks, 2 chunks and groups
    unsigned long long seq;             // r + 1, written last
    unsigned long long pad;
};

struct __align__(16) LoopResult {       // device -> host, one per slot
    double H[144], b[12], cost;
    long long count;                    // inliers (linearise) or hits (overlap)
    unsigned long long done;            // = seq once the fields above are complete
    unsigned long long pad;
};

struct LoopControl {                    // device memory, written by the host before each launch
    unsigned int item_head, item_tail, quit;
    unsigned int status;                // VGICP_ERR_TIMEOUT when a worker's own limit ran out
    unsigned long long next_req;        // first request the dispatcher waits for
};

struct LoopExit {                       // host-mapped
    int status;                         // device, at the end: VGICP_OK when asked to stop,
                                        // VGICP_ERR_TIMEOUT when the idle limit ran out
    int stop;                           // host: 1 asks the dispatcher to end
    unsigned long long next_req;        // device, at the end: first request not dispatched
};

struct __align__(16) LoopSlotState {    // device memory, one per slot
    PoseParam P;
    MapDesc map;
    FrameDesc frame;
    int32_t kind, n_items, chunk;
    unsigned int done_items;
    unsigned long long seq;
};

struct LoopArgs {
    const LoopRequest *req;             // device view of the mapped request ring
    LoopResult *res;                    // device view of the mapped result ring
    LoopExit *exit;                     // device view of the mapped exit record
    LoopControl *ctl;
    LoopSlotState *state;
    double *partials;                   // slots x kLoopMaxItems x 28
    long long *counts;                  // slots x kLoopMaxItems
    int2 *queue;                        // qcap entries (slot, chunk)
    int slots;
    unsigned int qcap;                  // power of two >= slots x kLoopMaxItems
    unsigned long long idle_ns, worker_ns;
};

void launch_request_loop(const LoopArgs &a, int num_sms, cudaStream_t st);

}  // namespace vg
