// vgicp_linearize_noalloc: the batched float32 linearisation with every
// intermediate buffer in one fixed, file-scope device array, so a call makes no
// device (or host) allocation.
//
// Some callers cannot allocate at call time: a mapping loop that fixes its
// device-memory footprint when it starts (so an optimiser iteration can never
// fail for lack of memory), or an application whose own allocator owns all
// device memory and must not be bypassed.  They keep their voxelmaps and frames
// in a context created up front, bring their own output buffers, and call this
// entry point instead of vgicp_linearize().
//
// The scratch array (kScratchBytes, about 4.5 MB) is loaded with the library
// and held on every GPU that loads it until the process exits.  Host code
// cannot use the array's name as a device address, so the first call on each
// device, with that device current, asks the runtime for the array's device
// address (cudaGetSymbolAddress) and keeps it; that first call should come
// before any stream capture.  Every call reuses the same array and finds the
// previous call's contents in it: each slot a call reads is written earlier in
// the same call, so nothing needs clearing, but calls whose work overlaps on the
// GPU (different streams, or different host threads) race on the array.
#include <mutex>

#include "kernels.cuh"
#include "vgicp.h"

namespace vg {
vgicp_status ctx_fail(::vgicp_ctx *ctx, vgicp_status s, const char *msg);
}

namespace {

using namespace vg;

constexpr int kMaxFactors = VGICP_NOALLOC_MAX_FACTORS;
constexpr int kMaxPoses = VGICP_NOALLOC_MAX_POSES;
constexpr int kMaxItems = VGICP_NOALLOC_MAX_ITEMS;
constexpr int kMaxDevices = 64;

constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffFactors = 0;
constexpr size_t kOffPoses = kOffFactors + al(sizeof(vgicp_factor) * kMaxFactors);
constexpr size_t kOffIdx = kOffPoses + al(sizeof(double) * 12 * kMaxPoses);
constexpr size_t kOffParams = kOffIdx + al(sizeof(int32_t) * 4 * kMaxFactors);
constexpr size_t kOffBegin = kOffParams + al(sizeof(PoseParam) * kMaxFactors);
constexpr size_t kOffItems = kOffBegin + al(sizeof(int32_t) * 2 * kMaxFactors);
constexpr size_t kOffPartials = kOffItems + al(sizeof(WorkItem) * kMaxItems);
constexpr size_t kOffInl = kOffPartials + al(sizeof(double) * 28 * kMaxItems);
constexpr size_t kOffFetch = kOffInl + al(sizeof(int64_t) * kMaxItems);
constexpr size_t kScratchBytes = kOffFetch + al(sizeof(int));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on `device` (current), looked up once.
cudaError_t scratch_address(int device, void **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

// One block: factor handles -> descriptor-table indices, then each factor's
// chunk count, an exclusive scan, the chunk work items and each factor's item
// range.
__global__ void k_noalloc_plan(const vgicp_factor *__restrict__ f, int n_f, const FrameDesc *__restrict__ frames,
                               int chunk, int32_t *__restrict__ idx, int32_t *__restrict__ item_range,
                               WorkItem *__restrict__ items)
{
    __shared__ int32_t s_scan[kMaxFactors];
    const int i = threadIdx.x;
    int32_t nchunks = 0;
    int64_t n = 0;
    int c = chunk;
    if (i < n_f) {
        const int32_t mi = (int32_t)(f[i].target & 0xffffffff), fi = (int32_t)(f[i].source & 0xffffffff);
        idx[4 * i + 0] = mi;
        idx[4 * i + 1] = fi;
        idx[4 * i + 2] = f[i].target_pose;
        idx[4 * i + 3] = f[i].source_pose;
        n = frames[fi].n;
        c = item_chunk(n, chunk);
        nchunks = (int32_t)((n + c - 1) / c);
    }
    s_scan[i] = nchunks;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const int32_t v = (i >= off) ? s_scan[i - off] : 0;
        __syncthreads();
        s_scan[i] += v;
        __syncthreads();
    }
    if (i < n_f) {
        const int32_t begin = s_scan[i] - nchunks;
        item_range[2 * i] = begin;
        item_range[2 * i + 1] = begin + nchunks;
        for (int32_t k = 0; k < nchunks; ++k) {
            WorkItem w;
            w.unit = i;
            w.start = (int64_t)k * c;
            w.count = (int32_t)((n - w.start < c) ? (n - w.start) : c);
            items[begin + k] = w;
        }
    }
}

}  // namespace

extern "C" vgicp_status vgicp_linearize_noalloc(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f,
                                                const double *poses, int64_t n_poses, double *H, double *b,
                                                double *cost, int64_t *inliers)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    CtxView v;
    if (!ctx_view(ctx, &v)) return ctx_fail(ctx, VGICP_ERR_INVALID_ARG, "linearize_noalloc: context not usable");
    // an error left by earlier, unrelated work on this thread is not this call's
    (void)cudaGetLastError();
    if (n_f < 0 || n_poses < 0 || (n_f > 0 && (!factors || !H || !b || !cost)) || (n_poses > 0 && !poses))
        return ctx_fail(ctx, VGICP_ERR_INVALID_ARG, "linearize_noalloc: null pointer or negative size");
    if (n_f > kMaxFactors || n_poses > kMaxPoses)
        return ctx_fail(ctx, VGICP_ERR_INVALID_ARG,
                        "linearize_noalloc: more than VGICP_NOALLOC_MAX_FACTORS factors or "
                        "VGICP_NOALLOC_MAX_POSES poses");
    if (n_f == 0) return VGICP_OK;
    int64_t n_items = 0;
    for (int64_t i = 0; i < n_f; ++i) {
        int64_t n = 0;
        if (!ctx_is_map(ctx, factors[i].target) || !ctx_frame_size(ctx, factors[i].source, &n))
            return ctx_fail(ctx, VGICP_ERR_NOT_FOUND, "linearize_noalloc: a factor names an unknown handle");
        if (factors[i].target_pose < 0 || factors[i].target_pose >= n_poses || factors[i].source_pose < 0 ||
            factors[i].source_pose >= n_poses)
            return ctx_fail(ctx, VGICP_ERR_INVALID_ARG, "linearize_noalloc: pose index out of range");
        const int c = item_chunk(n, v.chunk);
        n_items += (n + c - 1) / c;
    }
    if (n_items > kMaxItems)
        return ctx_fail(ctx, VGICP_ERR_INVALID_ARG,
                        "linearize_noalloc: the factors need more than VGICP_NOALLOC_MAX_ITEMS chunks");
    for (int64_t i = 0; i < n_poses * 12; ++i)
        if (!(poses[i] - poses[i] == 0.0))
            return ctx_fail(ctx, VGICP_ERR_INVALID_ARG, "linearize_noalloc: non-finite pose entry");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != v.device || dev < 0 || dev >= kMaxDevices)
        return ctx_fail(ctx, VGICP_ERR_CUDA, "linearize_noalloc: the context's device must be current");
    void *base = nullptr;
    cudaError_t e = scratch_address(dev, &base);
    if (e != cudaSuccess) return ctx_fail(ctx, VGICP_ERR_CUDA, cudaGetErrorString(e));
    char *s = (char *)base;
    vgicp_factor *d_f = (vgicp_factor *)(s + kOffFactors);
    double *d_poses = (double *)(s + kOffPoses);
    int32_t *d_idx = (int32_t *)(s + kOffIdx);
    PoseParam *d_params = (PoseParam *)(s + kOffParams);
    int32_t *d_begin = (int32_t *)(s + kOffBegin);
    WorkItem *d_items = (WorkItem *)(s + kOffItems);
    double *d_partials = (double *)(s + kOffPartials);
    int64_t *d_inl = (int64_t *)(s + kOffInl);
    int *d_fetch = (int *)(s + kOffFetch);
    e = cudaMemcpyAsync(d_f, factors, sizeof(vgicp_factor) * (size_t)n_f, cudaMemcpyHostToDevice, v.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_poses, poses, sizeof(double) * 12 * (size_t)n_poses, cudaMemcpyHostToDevice, v.stream);
    if (e != cudaSuccess) return ctx_fail(ctx, VGICP_ERR_CUDA, cudaGetErrorString(e));
    int threads = 32;
    while (threads < n_f) threads <<= 1;
    // the shared-memory map variant (6) needs per-map images made on demand;
    // here it runs as the default register variant, whose per-item arithmetic
    // and lane order are the same, so the results are too
    const int variant = v.variant == 6 ? 0 : v.variant;
    k_noalloc_plan<<<1, threads, 0, v.stream>>>(d_f, (int)n_f, v.d_frames, v.chunk, d_idx, d_begin, d_items);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        launch_prepare_factors(d_idx, (int)n_f, d_poses, v.d_maps, v.d_frames, v.linearize_cull, d_params,
                               v.stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        launch_linearize_f32(d_params, v.d_maps, v.d_frames, d_items, (int)n_items, d_partials, d_inl, d_fetch,
                             variant, v.blocks_per_sm, v.num_sms, v.compensated, v.neighbors, v.count_weighted,
                             v.stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        launch_reduce_finalize(d_params, d_begin, (int)n_f, d_partials, d_inl, H, b, cost, inliers, v.stream);
        e = cudaGetLastError();
    }
    ctx_count_launches(ctx, 3 + (n_items > 0));
    if (e != cudaSuccess) return ctx_fail(ctx, VGICP_ERR_CUDA, cudaGetErrorString(e));
    return VGICP_OK;
}
