// C ABI of the VGICP library: contexts, handles, device memory and the host
// side of every call declared in include/vgicp.h.  All arithmetic of the
// method runs in the kernels; this file validates arguments, owns memory,
// builds work lists and orders launches on the context stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "vgicp.h"

using namespace vg;

namespace {

struct Obj {
    enum Kind { FREE = 0, FRAME = 1, MAP = 2 } kind = FREE;
    uint32_t gen = 0;
    // frame
    int64_t n = 0;
    void *frame_mem = nullptr;
    size_t frame_bytes = 0;
    // map
    void *map_mem = nullptr;
    size_t map_bytes = 0;
    uint32_t cap = 0;
    double r = 0.0;
    bool img = false;   // shared-memory image made since the last build
};

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

// A cached work list for a factor set: device copies of the per-factor indices,
// the chunk items and each factor's first item.
struct Plan {
    std::vector<vgicp_factor> key;
    std::vector<int64_t> frame_n;
    int chunk = 0;
    int n_items = 0, n_units = 0;
    Buf idx, items, item_range, units;
};

constexpr int kMaxLanes = 4;

// Everything one stream of work needs on its own: the stream, the work lists
// and the scratch buffers.  Handles, descriptor tables and options are shared
// by all lanes of a context.
struct Lane {
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    Buf ws_poses, ws_params, ws_partials, ws_inl, ws_out, ws_f64, ws_ticket, ws_counts, ws_stage;
    Buf ws_bunits, ws_bitems, ws_slot_of_point, ws_acc, ws_vid_of_slot, ws_slot_of_vid;
    Buf ws_pairs, ws_fidx, ws_midx, ws_chunks, ws_export_keys, ws_export_rec, ws_counter, ws_descs, ws_tune, ws_knn;
    Buf ws_fetch, ws_items, ws_img, ws_rec, ws_order;
    Plan plan;
    int64_t last_matrix_pairs = 0;   // pairs of the last overlap matrix (params kept in ws_pairs)
    // pinned staging for host -> device copies: two arenas used in turn, each
    // with an event after its latest copy, so copies never wait for the stream
    struct Arena {
        char *p = nullptr;
        char *dp = nullptr;   // the same memory as the device addresses it
        size_t cap = 0, off = 0;
        cudaEvent_t ev = nullptr;
        bool pending = false;
    } arena[2];
    int arena_cur = 0;
    cudaEvent_t big_copy = nullptr;   // after this lane's last large host -> device copy
    bool big_copy_pending = false;
    char *d2h_stage = nullptr;   // page-locked landing buffer for small results
    size_t d2h_cap = 0;
    // event pairs around the hot kernels' launches (vgicp_kernel_timing)
    struct KTimer {
        std::vector<cudaEvent_t> begin, end;
        int used = 0;
    } ktimer[3];
};

}  // namespace

struct vgicp_ctx {
    int device = 0;
    int num_sms = 148;
    vgicp_options opt{};
    std::string err;
    std::vector<Obj> objs;
    std::vector<uint32_t> free_idx;
    // per descriptor index: an event recorded on the lane that released the
    // index (after the work that lane had enqueued, which may still read the
    // index's descriptor), waited for by the lane that takes the index again
    std::vector<cudaEvent_t> idx_ev;
    std::vector<uint8_t> idx_ev_set;
    int64_t bytes_in_use = 0;
    int64_t launches = 0;
    // descriptor tables (device) and host mirrors
    MapDesc *d_maps = nullptr;
    FrameDesc *d_frames = nullptr;
    std::vector<MapDesc> h_maps;
    std::vector<FrameDesc> h_frames;
    size_t tab_cap = 0;
    Lane lanes[kMaxLanes];
    int lane = 0;
};

// the current lane's stream and buffers
#define LN (ctx->lanes[ctx->lane])

namespace {


vgicp_status fail(vgicp_ctx *c, vgicp_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define CU(call)                                                                                            \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess)                                                                              \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? VGICP_ERR_OOM : VGICP_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                                 \
    } while (0)

#define CHECK_LAUNCH()                                                                                      \
    do {                                                                                                    \
        cudaError_t e_ = cudaGetLastError();                                                                \
        if (e_ != cudaSuccess)                                                                              \
            return fail(ctx, VGICP_ERR_CUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__,  \
                        __LINE__);                                                                          \
    } while (0)

#define TRY(expr)                               \
    do {                                        \
        vgicp_status s_ = (expr);               \
        if (s_ != VGICP_OK) return s_;          \
    } while (0)

vgicp_status ensure(vgicp_ctx *ctx, Buf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return VGICP_OK;
    if (b.p) CU(cudaFreeAsync(b.p, LN.stream));
    b.p = nullptr;
    b.bytes = 0;
    size_t nb = std::max(bytes, b.bytes * 3 / 2);
    CU(cudaMallocAsync(&b.p, nb, LN.stream));
    b.bytes = nb;
    return VGICP_OK;
}

void free_buf(vgicp_ctx *ctx, Buf &b)
{
    if (b.p) cudaFreeAsync(b.p, LN.stream);
    b.p = nullptr;
    b.bytes = 0;
}

// Host -> device copy in stream order that returns without waiting for the
// stream: the bytes go through a pinned staging arena of the lane (a copy from
// pageable memory may first wait for the work queued before it).  An arena is
// reused only after every copy from it has run; very large copies go direct.
constexpr size_t kArenaMaxCopy = (size_t)4 << 20, kCopyPiece = (size_t)8 << 20;

bool page_locked(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// Small uploads go through the lane's page-locked arena.  The copy engine
// serves the work of several streams in submission order, so while another
// lane's large copy is in flight a cudaMemcpyAsync here would wait for all of
// it; then the upload is a kernel that reads the arena over the bus instead.
// Otherwise the copy engine takes it (a kernel could in turn wait for SMs that
// another lane's persistent kernel holds).
__global__ void k_upload(unsigned char *__restrict__ dst, const unsigned char *__restrict__ src, size_t bytes)
{
    const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    if ((((uintptr_t)dst | (uintptr_t)src) & 15) == 0) {
        const size_t n16 = bytes >> 4;
        for (size_t i = tid; i < n16; i += stride) ((uint4 *)dst)[i] = ((const uint4 *)src)[i];
        for (size_t i = (n16 << 4) + tid; i < bytes; i += stride) dst[i] = src[i];
    } else {
        for (size_t i = tid; i < bytes; i += stride) dst[i] = src[i];
    }
}

// Whether a large host -> device copy issued on another lane may still be running.
bool other_lane_copying(vgicp_ctx *ctx)
{
    bool busy = false;
    for (int l = 0; l < kMaxLanes; ++l) {
        Lane &L = ctx->lanes[l];
        if (l == ctx->lane || !L.big_copy_pending) continue;
        const cudaError_t q = cudaEventQuery(L.big_copy);
        if (q == cudaSuccess) {
            L.big_copy_pending = false;
        } else {
            if (cudaPeekAtLastError() == q) cudaGetLastError();   // "not ready" is a state, not a failure
            busy = true;
        }
    }
    return busy;
}

vgicp_status h2d(vgicp_ctx *ctx, void *dst, const void *src, size_t bytes)
{
    if (bytes == 0) return VGICP_OK;
    if (bytes >= 65536 && page_locked(src)) {
        // page-locked memory is copied directly, in pieces
        for (size_t o = 0; o < bytes; o += kCopyPiece)
            CU(cudaMemcpyAsync((char *)dst + o, (const char *)src + o, std::min(kCopyPiece, bytes - o),
                               cudaMemcpyHostToDevice, LN.stream));
        if (!LN.big_copy) CU(cudaEventCreateWithFlags(&LN.big_copy, cudaEventDisableTiming));
        CU(cudaEventRecord(LN.big_copy, LN.stream));
        LN.big_copy_pending = true;
        return VGICP_OK;
    }
    if (bytes > kArenaMaxCopy) {
        // large pageable copies: the driver stages them itself
        CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, LN.stream));
        return VGICP_OK;
    }
    Lane::Arena *A = &LN.arena[LN.arena_cur];
    if (A->off + bytes > A->cap) {
        LN.arena_cur ^= 1;
        A = &LN.arena[LN.arena_cur];
        if (A->pending) CU(cudaEventSynchronize(A->ev));
        A->pending = false;
        A->off = 0;
        if (A->cap < bytes) {
            if (A->p) CU(cudaFreeHost(A->p));
            A->p = nullptr;
            A->cap = 0;
            const size_t cap = std::max<size_t>(std::max<size_t>(bytes * 2, (size_t)4 << 20), A->cap * 2);
            CU(cudaMallocHost((void **)&A->p, cap));
            CU(cudaHostGetDevicePointer((void **)&A->dp, A->p, 0));
            A->cap = cap;
        }
        if (!A->ev) CU(cudaEventCreateWithFlags(&A->ev, cudaEventDisableTiming));
    }
    const size_t at = A->off;
    A->off = (A->off + bytes + 255) & ~(size_t)255;
    std::memcpy(A->p + at, src, bytes);
    if (other_lane_copying(ctx)) {
        const int grid = (int)std::min<size_t>((bytes + 4095) / 4096, (size_t)ctx->num_sms * 2);
        k_upload<<<grid, 256, 0, LN.stream>>>((unsigned char *)dst, (const unsigned char *)(A->dp + at), bytes);
        ctx->launches += 1;
        CHECK_LAUNCH();
    } else {
        CU(cudaMemcpyAsync(dst, A->p + at, bytes, cudaMemcpyHostToDevice, LN.stream));
    }
    CU(cudaEventRecord(A->ev, LN.stream));
    A->pending = true;
    return VGICP_OK;
}

// A contiguous device block [src, src + sum of bytes) read back into k host
// destinations in order (a null destination skips its piece), then the lane is
// synchronised.  Small results land in a page-locked buffer of the lane with
// one copy and are spread by the host: a copy into pageable memory costs a
// driver round trip each.
constexpr size_t kD2HStageMax = (size_t)256 << 10;

vgicp_status d2h_pieces(vgicp_ctx *ctx, const void *src, void *const *dst, const size_t *bytes, int k)
{
    size_t total = 0;
    for (int i = 0; i < k; ++i) total += bytes[i];
    if (total == 0) return VGICP_OK;
    if (total <= kD2HStageMax) {
        if (LN.d2h_cap < total) {
            if (LN.d2h_stage) CU(cudaFreeHost(LN.d2h_stage));
            LN.d2h_stage = nullptr;
            LN.d2h_cap = 0;
            CU(cudaMallocHost((void **)&LN.d2h_stage, kD2HStageMax));
            LN.d2h_cap = kD2HStageMax;
        }
        CU(cudaMemcpyAsync(LN.d2h_stage, src, total, cudaMemcpyDeviceToHost, LN.stream));
        CU(cudaStreamSynchronize(LN.stream));
        size_t o = 0;
        for (int i = 0; i < k; ++i) {
            if (dst[i] && bytes[i]) std::memcpy(dst[i], LN.d2h_stage + o, bytes[i]);
            o += bytes[i];
        }
        return VGICP_OK;
    }
    size_t o = 0;
    for (int i = 0; i < k; ++i) {
        if (dst[i] && bytes[i])
            CU(cudaMemcpyAsync(dst[i], (const char *)src + o, bytes[i], cudaMemcpyDeviceToHost, LN.stream));
        o += bytes[i];
    }
    CU(cudaStreamSynchronize(LN.stream));
    return VGICP_OK;
}

// Event pair around one launch of hot kernel `id` on the current lane; -1 when
// the lane's record is full (1,024 launches since the last reset).
constexpr int kMaxTimed = 1024;

int ktimer_begin(vgicp_ctx *ctx, int id)
{
    Lane::KTimer &K = LN.ktimer[id];
    if (K.used >= kMaxTimed) return -1;
    if (K.used == (int)K.begin.size()) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
            if (a) cudaEventDestroy(a);
            cudaGetLastError();
            return -1;
        }
        K.begin.push_back(a);
        K.end.push_back(b);
    }
    if (cudaEventRecord(K.begin[K.used], LN.stream) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return K.used++;
}

void ktimer_end(vgicp_ctx *ctx, int id, int slot)
{
    if (slot < 0) return;
    if (cudaEventRecord(LN.ktimer[id].end[slot], LN.stream) != cudaSuccess) cudaGetLastError();
}

template <class T>
vgicp_status upload(vgicp_ctx *ctx, Buf &b, const T *src, size_t count)
{
    TRY(ensure(ctx, b, count * sizeof(T)));
    return h2d(ctx, b.p, src, count * sizeof(T));
}

inline int64_t make_handle(uint32_t idx, uint32_t gen) { return ((int64_t)gen << 32) | (int64_t)idx; }

Obj *lookup(vgicp_ctx *ctx, int64_t h, Obj::Kind kind, uint32_t *idx_out = nullptr)
{
    if (h < 0) return nullptr;
    const uint32_t idx = (uint32_t)(h & 0xffffffff), gen = (uint32_t)(h >> 32);
    if (idx >= ctx->objs.size()) return nullptr;
    Obj &o = ctx->objs[idx];
    if (o.kind != kind || o.gen != gen) return nullptr;
    if (idx_out) *idx_out = idx;
    return &o;
}

vgicp_status grow_tables(vgicp_ctx *ctx, size_t need)
{
    if (need <= ctx->tab_cap) return VGICP_OK;
    // other lanes may be reading or writing the current tables
    for (int l = 0; l < kMaxLanes; ++l)
        if (l != ctx->lane && ctx->lanes[l].stream) CU(cudaStreamSynchronize(ctx->lanes[l].stream));
    size_t cap = std::max<size_t>(64, ctx->tab_cap);
    while (cap < need) cap *= 2;
    MapDesc *nm = nullptr;
    FrameDesc *nf = nullptr;
    CU(cudaMallocAsync((void **)&nm, cap * sizeof(MapDesc), LN.stream));
    CU(cudaMallocAsync((void **)&nf, cap * sizeof(FrameDesc), LN.stream));
    CU(cudaMemsetAsync(nm, 0, cap * sizeof(MapDesc), LN.stream));
    CU(cudaMemsetAsync(nf, 0, cap * sizeof(FrameDesc), LN.stream));
    if (ctx->tab_cap) {
        CU(cudaMemcpyAsync(nm, ctx->d_maps, ctx->tab_cap * sizeof(MapDesc), cudaMemcpyDeviceToDevice, LN.stream));
        CU(cudaMemcpyAsync(nf, ctx->d_frames, ctx->tab_cap * sizeof(FrameDesc), cudaMemcpyDeviceToDevice,
                           LN.stream));
        CU(cudaFreeAsync(ctx->d_maps, LN.stream));
        CU(cudaFreeAsync(ctx->d_frames, LN.stream));
    }
    // the new tables are complete before any lane's later work can read them
    CU(cudaStreamSynchronize(LN.stream));
    ctx->d_maps = nm;
    ctx->d_frames = nf;
    ctx->tab_cap = cap;
    ctx->h_maps.resize(cap);
    ctx->h_frames.resize(cap);
    return VGICP_OK;
}

vgicp_status new_obj(vgicp_ctx *ctx, Obj::Kind kind, uint32_t *idx)
{
    uint32_t i;
    if (!ctx->free_idx.empty()) {
        i = ctx->free_idx.back();
        ctx->free_idx.pop_back();
        // the lane that released i may still have work queued that reads the
        // descriptor at i: this lane's writes to it come after that work
        if (i < ctx->idx_ev_set.size() && ctx->idx_ev_set[i]) {
            ctx->idx_ev_set[i] = 0;
            CU(cudaStreamWaitEvent(LN.stream, ctx->idx_ev[i], 0));
        }
    } else {
        i = (uint32_t)ctx->objs.size();
        ctx->objs.emplace_back();
    }
    TRY(grow_tables(ctx, ctx->objs.size()));
    Obj &o = ctx->objs[i];
    o.kind = kind;
    o.gen += 1;
    *idx = i;
    return VGICP_OK;
}

vgicp_status budget_check(vgicp_ctx *ctx, int64_t extra)
{
    if (ctx->opt.hbm_budget_bytes > 0 && ctx->bytes_in_use + extra > ctx->opt.hbm_budget_bytes)
        return fail(ctx, VGICP_ERR_BUDGET, "device budget %lld B exceeded (in use %lld B, requested %lld B)",
                    (long long)ctx->opt.hbm_budget_bytes, (long long)ctx->bytes_in_use, (long long)extra);
    return VGICP_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device bytes of a frame of n points: pa, pb, pc, statistics, chunk boxes,
// group boxes, and the storage permutation of a spatially ordered frame.
size_t group_box_bytes(int64_t n) { return align256((size_t)((n + kGroup - 1) / kGroup) * 24); }
size_t frame_bytes(int64_t n, bool ordered)
{
    return align256((size_t)n * 16) * 2 + align256((size_t)n * 4) + 256 + 1024 + group_box_bytes(n) +
           (ordered ? align256((size_t)n * 4) : 0);
}

// Allocate a frame handle of n points and fill its host descriptor (the
// device copy of the descriptor and the data are the caller's business).
vgicp_status alloc_frame(vgicp_ctx *ctx, int64_t n, uint32_t *out_idx)
{
    const bool ordered = ctx->opt.frame_order != 0 && n > 1;
    const size_t o_pb = align256((size_t)n * 16), o_pc = o_pb + align256((size_t)n * 16);
    const size_t o_st = o_pc + align256((size_t)n * 4), o_cb = o_st + 256, o_gb = o_cb + 1024;
    const size_t o_pm = o_gb + group_box_bytes(n);
    const size_t bytes = o_pm + (ordered ? align256((size_t)n * 4) : 0);
    TRY(budget_check(ctx, (int64_t)bytes));
    uint32_t idx;
    TRY(new_obj(ctx, Obj::FRAME, &idx));
    Obj &o = ctx->objs[idx];
    char *base = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&base, bytes, LN.stream);
    if (e != cudaSuccess) {
        o.kind = Obj::FREE;
        ctx->free_idx.push_back(idx);
        return fail(ctx, VGICP_ERR_OOM, "frame allocation of %zu B failed: %s", bytes, cudaGetErrorString(e));
    }
    o.n = n;
    o.frame_mem = base;
    o.frame_bytes = bytes;
    ctx->bytes_in_use += (int64_t)bytes;
    FrameDesc &f = ctx->h_frames[idx];
    f.pa = (const float4 *)base;
    f.pb = (const float4 *)(base + o_pb);
    f.pc = (const float *)(base + o_pc);
    f.stats = (const float *)(base + o_st);
    f.cbox = (const float *)(base + o_cb);
    f.perm = ordered ? (const int32_t *)(base + o_pm) : nullptr;
    f.gbox = (const float *)(base + o_gb);
    f.n = n;
    f.cshift = 10;
    while (((int64_t)kMaxCullChunks << f.cshift) < n) ++f.cshift;
    f.nchunks = (int32_t)((n + ((int64_t)1 << f.cshift) - 1) >> f.cshift);
    *out_idx = idx;
    return VGICP_OK;
}

uint32_t map_capacity(int64_t n)
{
    int64_t want = std::max<int64_t>(16, n + n / 2 + 1);
    uint32_t cap = 16;
    while ((int64_t)cap < want) cap <<= 1;
    return cap;
}

bool is_pow2_res(double r)
{
    int e;
    return std::frexp(r, &e) == 0.5;
}

size_t map_bytes(uint32_t cap);

void fill_map_desc(MapDesc &m, char *base, uint32_t cap, double r)
{
    m.keys = (uint64_t *)base;
    m.rec = (VoxelRec *)(base + align256((size_t)cap * 8));
    m.ckeys = (uint32_t *)(base + align256((size_t)cap * 8) + align256((size_t)cap * sizeof(VoxelRec)));
    m.img = (unsigned char *)(base + align256((size_t)cap * 8) + align256((size_t)cap * sizeof(VoxelRec)) +
                              align256((size_t)cap * 4));
    m.coarse = (uint32_t *)(base + map_bytes(cap) - 256 - align256(kCoarseWords * 4));
    m.kbox = (int32_t *)(base + map_bytes(cap) - 256 + 16);
    m.cmeta = (int32_t *)(base + map_bytes(cap) - 256 + 48);
    m.mask = cap - 1;
    uint32_t l = 0;
    while ((1u << l) < cap) ++l;
    m.log2cap = l;
    m.r = r;
    m.inv_r = 1.0 / r;
    m.r_h = (float)r;
    m.r_l = (float)(r - (double)m.r_h);
    m.inv_rf = (float)m.inv_r;
    m.pow2 = is_pow2_res(r) ? 1 : 0;
}

size_t map_bytes(uint32_t cap)
{
    return align256((size_t)cap * 8) + align256((size_t)cap * sizeof(VoxelRec)) + align256((size_t)cap * 4) +
           align256(kImgMaxBytes) + align256(kCoarseWords * 4) + 256;
}

uint32_t *map_nvox_ptr(const Obj &o) { return (uint32_t *)((char *)o.map_mem + o.map_bytes - 256); }

// Build voxelmaps for frame indices fidx[] into map indices midx[] (already allocated).
vgicp_status run_build(vgicp_ctx *ctx, const std::vector<uint32_t> &fidx, const std::vector<uint32_t> &midx)
{
    const int nu = (int)fidx.size();
    std::vector<BuildUnit> units(nu);
    std::vector<int64_t> prefix(nu + 1, 0);
    std::vector<WorkItem> items;
    int64_t pts = 0;
    const int chunk = 2048;
    for (int u = 0; u < nu; ++u) {
        const Obj &fo = ctx->objs[fidx[u]];
        const Obj &mo = ctx->objs[midx[u]];
        units[u].map = (int32_t)midx[u];
        units[u].frame = (int32_t)fidx[u];
        units[u].point_base = pts;
        units[u].slot_base = prefix[u];
        units[u].n_voxels = map_nvox_ptr(mo);
        units[u].pad = 0;
        prefix[u + 1] = prefix[u] + mo.cap;
        for (int64_t s = 0; s < fo.n; s += chunk) {
            WorkItem w;
            w.unit = u;
            w.start = s;
            w.count = (int32_t)std::min<int64_t>(chunk, fo.n - s);
            items.push_back(w);
        }
        pts += fo.n;
    }
    TRY(upload(ctx, LN.ws_bunits, units.data(), units.size()));
    TRY(upload(ctx, LN.ws_bitems, items.data(), items.size()));
    TRY(ensure(ctx, LN.ws_slot_of_point, (size_t)pts * 4));
    TRY(ensure(ctx, LN.ws_acc, (size_t)pts * 80));
    TRY(ensure(ctx, LN.ws_vid_of_slot, (size_t)prefix[nu] * 4));
    TRY(ensure(ctx, LN.ws_slot_of_vid, (size_t)pts * 4));
    BuildScratch scr;
    scr.slot_of_point = (int32_t *)LN.ws_slot_of_point.p;
    scr.acc = (int64_t *)LN.ws_acc.p;
    scr.vid_of_slot = (int32_t *)LN.ws_vid_of_slot.p;
    scr.slot_of_vid = (int32_t *)LN.ws_slot_of_vid.p;
    const int grid = std::max(1, std::min<int>((int)items.size(), ctx->num_sms * 8));
    const int kt = ktimer_begin(ctx, VGICP_KERNEL_VOXELMAP_BUILD);
    launch_voxelmap_build(ctx->d_maps, ctx->d_frames, (const BuildUnit *)LN.ws_bunits.p, nu,
                          (const WorkItem *)LN.ws_bitems.p, (int)items.size(),
                          scr, grid, LN.stream);
    ktimer_end(ctx, VGICP_KERNEL_VOXELMAP_BUILD, kt);
    ctx->launches += 1 + (items.empty() ? 0 : 3);
    CHECK_LAUNCH();
    return VGICP_OK;
}

// Make sure map object idx has capacity for n points at resolution r; *changed
// says whether its descriptor differs from the one in the device table.
vgicp_status prepare_map(vgicp_ctx *ctx, uint32_t idx, int64_t n, double r, bool *changed)
{
    Obj &o = ctx->objs[idx];
    const uint32_t cap = map_capacity(n);
    if (o.map_mem == nullptr || o.cap < cap) {
        const size_t bytes = map_bytes(cap);
        TRY(budget_check(ctx, (int64_t)bytes - (int64_t)o.map_bytes));
        if (o.map_mem) {
            CU(cudaFreeAsync(o.map_mem, LN.stream));
            ctx->bytes_in_use -= (int64_t)o.map_bytes;
            o.map_mem = nullptr;
        }
        CU(cudaMallocAsync(&o.map_mem, bytes, LN.stream));
        o.map_bytes = bytes;
        o.cap = cap;
        ctx->bytes_in_use += (int64_t)bytes;
    }
    o.r = r;
    o.img = false;
    MapDesc d{};
    fill_map_desc(d, (char *)o.map_mem, o.cap, r);
    *changed = std::memcmp(&d, &ctx->h_maps[idx], sizeof(MapDesc)) != 0;
    ctx->h_maps[idx] = d;
    return VGICP_OK;
}

bool valid_res(double r) { return std::isfinite(r) && r > 0.0 && r < 1e30; }

bool finite_pose(const double *T)
{
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(T[i])) return false;
    return true;
}

vgicp_status read_nvox(vgicp_ctx *ctx, const Obj &o, int64_t *n)
{
    uint32_t v = 0;
    CU(cudaMemcpyAsync(&v, map_nvox_ptr(o), 4, cudaMemcpyDeviceToHost, LN.stream));
    CU(cudaStreamSynchronize(LN.stream));
    *n = v;
    return VGICP_OK;
}

int default_chunk(const vgicp_options &o) { return o.chunk_points > 0 ? o.chunk_points : 2048; }
int neighbor_count(const vgicp_options &o) { return o.neighbors > 1 ? o.neighbors : 1; }
// chunk culling tests the target's voxel box, so it holds for the containing voxel only
// Culling level handed to the pair preparation: 0 none, 1 pairs and cull
// chunks, 2 also groups of kGroup points against the coarse occupancy.
int cull_level(int on, const vgicp_options &o) { return on ? (o.group_cull ? 2 : 1) : 0; }
int lin_cull(const vgicp_options &o) { return neighbor_count(o) == 1 ? cull_level(o.linearize_cull, o) : 0; }
int ov_cull(const vgicp_options &o) { return cull_level(o.overlap_cull, o); }
// variant 6: the shared-memory map path (single-voxel, unweighted association)
bool uses_img(const vgicp_options &o) { return o.linearize_variant == 6 && neighbor_count(o) == 1 && !o.count_weighted; }

// Shared-memory images of a factor set's maps that have none since their last
// build, made on the lane's stream ahead of the linearisation that reads them.
vgicp_status ensure_images(vgicp_ctx *ctx, const std::vector<int32_t> &idx, int64_t n_f)
{
    std::vector<int32_t> todo;
    for (int64_t i = 0; i < n_f; ++i) {
        Obj &o = ctx->objs[idx[4 * i]];
        if (!o.img) {
            o.img = true;
            todo.push_back(idx[4 * i]);
        }
    }
    if (todo.empty()) return VGICP_OK;
    TRY(upload(ctx, LN.ws_img, todo.data(), todo.size()));
    launch_map_images(ctx->d_maps, (const int32_t *)LN.ws_img.p, (int)todo.size(), ctx->num_sms, LN.stream);
    ctx->launches += 1;
    CHECK_LAUNCH();
    return VGICP_OK;
}

// Descriptor-table indices of a factor set (map, frame, target pose, source
// pose per factor), after checking handles, pose indices and pose entries.
vgicp_status factor_indices(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f, const double *poses,
                            int64_t n_poses, std::vector<int32_t> &idx)
{
    if (n_f > (1 << 30)) return fail(ctx, VGICP_ERR_INVALID_ARG, "too many factors");
    idx.resize((size_t)n_f * 4);
    for (int64_t i = 0; i < n_f; ++i) {
        uint32_t mi, fi;
        if (!lookup(ctx, factors[i].target, Obj::MAP, &mi))
            return fail(ctx, VGICP_ERR_NOT_FOUND, "factor %lld: map handle %lld not found", (long long)i,
                        (long long)factors[i].target);
        if (!lookup(ctx, factors[i].source, Obj::FRAME, &fi))
            return fail(ctx, VGICP_ERR_NOT_FOUND, "factor %lld: frame handle %lld not found", (long long)i,
                        (long long)factors[i].source);
        if (factors[i].target_pose < 0 || factors[i].target_pose >= n_poses || factors[i].source_pose < 0 ||
            factors[i].source_pose >= n_poses)
            return fail(ctx, VGICP_ERR_INVALID_ARG, "factor %lld: pose index out of range", (long long)i);
        idx[4 * i + 0] = (int32_t)mi;
        idx[4 * i + 1] = (int32_t)fi;
        idx[4 * i + 2] = factors[i].target_pose;
        idx[4 * i + 3] = factors[i].source_pose;
    }
    for (int64_t i = 0; i < n_poses * 12; ++i)
        if (!std::isfinite(poses[i])) return fail(ctx, VGICP_ERR_INVALID_ARG, "non-finite pose entry");
    return VGICP_OK;
}

// Work items of a factor set: each factor's points in chunks of `chunk`, the
// chunks of one factor contiguous, and factors grouped by target voxelmap (then
// by source frame) so that the warps running at any moment share few maps and
// their voxel records stay in L2.  range[2 f], range[2 f + 1] delimit factor f's
// items.  The order changes no sum: each factor's chunks are reduced in chunk
// order whatever their position in the list.
// Work units of the shared-memory map path: runs of at most kUnitItems
// consecutive items with the same target map, (map, first item, end item, 0).
constexpr int kUnitItems = 32;

void build_units(const std::vector<int32_t> &idx, const std::vector<WorkItem> &items, std::vector<int4> &units)
{
    units.clear();
    size_t b = 0;
    while (b < items.size()) {
        const int32_t map = idx[4 * items[b].unit];
        size_t e = b + 1;
        while (e < items.size() && e - b < (size_t)kUnitItems && idx[4 * items[e].unit] == map) ++e;
        units.push_back(make_int4(map, (int)b, (int)e, 0));
        b = e;
    }
}

void build_items(const std::vector<int32_t> &idx, const std::vector<int64_t> &frame_n, int chunk,
                 std::vector<WorkItem> &items, std::vector<int32_t> &range)
{
    const int64_t n_f = (int64_t)frame_n.size();
    std::vector<int32_t> order((size_t)n_f);
    for (int64_t i = 0; i < n_f; ++i) order[i] = (int32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        if (idx[4 * a] != idx[4 * b]) return idx[4 * a] < idx[4 * b];
        return idx[4 * a + 1] < idx[4 * b + 1];
    });
    items.clear();
    range.assign((size_t)n_f * 2, 0);
    for (int32_t i : order) {
        const int64_t n = frame_n[i];
        const int c = item_chunk(n, chunk);
        range[2 * i] = (int32_t)items.size();
        for (int64_t s = 0; s < n; s += c) {
            WorkItem w;
            w.unit = i;
            w.start = s;
            w.count = (int32_t)std::min<int64_t>(c, n - s);
            items.push_back(w);
        }
        range[2 * i + 1] = (int32_t)items.size();
    }
}

// Work list for a factor set (cached while the set and the chunk size stay the same).
vgicp_status get_plan(vgicp_ctx *ctx, const vgicp_factor *f, int64_t n_f, const std::vector<int32_t> &idx)
{
    Plan &P = LN.plan;
    const int chunk = default_chunk(ctx->opt);
    bool same = P.chunk == chunk && (int64_t)P.key.size() == n_f &&
                std::memcmp(P.key.data(), f, sizeof(vgicp_factor) * (size_t)n_f) == 0;
    if (same) {
        for (int64_t i = 0; i < n_f && same; ++i) same = P.frame_n[i] == ctx->objs[idx[4 * i + 1]].n;
    }
    if (same) {
        // descriptor indices are embedded in the cached idx array; handles are
        // validated by the caller, so the cached copy is still exact
        return VGICP_OK;
    }
    P.frame_n.resize(n_f);
    for (int64_t i = 0; i < n_f; ++i) P.frame_n[i] = ctx->objs[idx[4 * i + 1]].n;
    std::vector<WorkItem> items;
    std::vector<int32_t> range;
    build_items(idx, P.frame_n, chunk, items, range);
    std::vector<int4> units;
    build_units(idx, items, units);
    TRY(upload(ctx, P.idx, idx.data(), idx.size()));
    TRY(upload(ctx, P.items, items.data(), items.size()));
    TRY(upload(ctx, P.item_range, range.data(), range.size()));
    TRY(upload(ctx, P.units, units.data(), units.size()));
    P.n_units = (int)units.size();
    P.key.assign(f, f + n_f);
    P.chunk = chunk;
    P.n_items = (int)items.size();
    return VGICP_OK;
}


}  // namespace

extern "C" {

vgicp_status vgicp_options_default(vgicp_options *opt)
{
    if (!opt) return VGICP_ERR_INVALID_ARG;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = VGICP_PREC_F32;
    opt->chunk_points = 2048;
    opt->neighbors = 1;
    opt->linearize_variant = 0;
    opt->blocks_per_sm = 0;
    opt->hbm_budget_bytes = 0;
    opt->overlap_cull = 1;
    opt->group_cull = 1;
    opt->linearize_cull = 1;
    opt->frame_order = 2;
    return VGICP_OK;
}

static vgicp_status check_options(vgicp_ctx *ctx, const vgicp_options *o)
{
    if (o->precision != VGICP_PREC_F32 && o->precision != VGICP_PREC_F64 && o->precision != VGICP_PREC_F32_COMP)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "precision must be VGICP_PREC_F32, VGICP_PREC_F64 or VGICP_PREC_F32_COMP");
    if (o->chunk_points < 0 || (o->chunk_points % 32) != 0)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "chunk_points must be a non-negative multiple of 32");
    if (o->neighbors != 0 && o->neighbors != 1 && o->neighbors != 7 && o->neighbors != 27)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "neighbors must be 1, 7 or 27");
    if (o->count_weighted != 0 && o->count_weighted != 1)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "count_weighted must be 0 or 1");
    if (o->linearize_variant < 0 || o->linearize_variant > 6)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "linearize_variant must be in 0..6");
    if (o->blocks_per_sm < 0 || o->hbm_budget_bytes < 0)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "blocks_per_sm and hbm_budget_bytes must be >= 0");
    if (o->overlap_cull != 0 && o->overlap_cull != 1)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "overlap_cull must be 0 or 1");
    if (o->group_cull != 0 && o->group_cull != 1)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "group_cull must be 0 or 1");
    if (o->frame_order < 0 || o->frame_order > 2)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "frame_order must be 0, 1 or 2");
    if (o->linearize_cull != 0 && o->linearize_cull != 1)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "linearize_cull must be 0 or 1");
    return VGICP_OK;
}

vgicp_status vgicp_create(vgicp_ctx **out, const vgicp_options *opt, void *cuda_stream)
{
    if (!out) return VGICP_ERR_INVALID_ARG;
    *out = nullptr;
    vgicp_ctx *ctx = new vgicp_ctx();
    vgicp_options_default(&ctx->opt);
    if (opt) {
        vgicp_status s = check_options(ctx, opt);
        if (s != VGICP_OK) { delete ctx; return s; }
        ctx->opt = *opt;
    }
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess && !cuda_stream) e = cudaStreamCreateWithFlags(&LN.own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        cudaMemPool_t pool;
        e = cudaDeviceGetDefaultMemPool(&pool, ctx->device);
        if (e == cudaSuccess) {
            uint64_t thr = ~0ull;
            e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    if (e != cudaSuccess) {
        delete ctx;
        return VGICP_ERR_CUDA;
    }
    LN.stream = cuda_stream ? (cudaStream_t)cuda_stream : LN.own_stream;
    *out = ctx;
    return VGICP_OK;
}

vgicp_status vgicp_destroy(vgicp_ctx *ctx)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    // every lane's work ends before the memory it may read is freed
    for (int l = 0; l < kMaxLanes; ++l)
        if (ctx->lanes[l].stream) cudaStreamSynchronize(ctx->lanes[l].stream);
    for (cudaEvent_t ev : ctx->idx_ev)
        if (ev) cudaEventDestroy(ev);
    ctx->lane = 0;
    for (Obj &o : ctx->objs) {
        if (o.frame_mem) cudaFreeAsync(o.frame_mem, LN.stream);
        if (o.map_mem) cudaFreeAsync(o.map_mem, LN.stream);
    }
    if (ctx->d_maps) cudaFreeAsync(ctx->d_maps, LN.stream);
    if (ctx->d_frames) cudaFreeAsync(ctx->d_frames, LN.stream);
    cudaError_t e = cudaSuccess;
    for (int l = kMaxLanes - 1; l >= 0; --l) {
        ctx->lane = l;
        if (!LN.stream) continue;
        Buf *bufs[] = {&LN.ws_poses, &LN.ws_params, &LN.ws_partials, &LN.ws_inl, &LN.ws_out, &LN.ws_f64,
                       &LN.ws_ticket, &LN.ws_counts, &LN.ws_stage, &LN.ws_bunits, &LN.ws_bitems,
                       &LN.ws_slot_of_point, &LN.ws_acc, &LN.ws_vid_of_slot,
                       &LN.ws_slot_of_vid, &LN.ws_img, &LN.ws_pairs, &LN.ws_fidx, &LN.ws_midx, &LN.ws_chunks,
                       &LN.ws_export_keys, &LN.ws_export_rec, &LN.ws_counter, &LN.ws_descs, &LN.ws_tune,
                       &LN.ws_knn, &LN.plan.idx, &LN.plan.items, &LN.plan.item_range, &LN.plan.units, &LN.ws_fetch,
                       &LN.ws_items, &LN.ws_rec, &LN.ws_order};
        for (Buf *b : bufs) free_buf(ctx, *b);
        const cudaError_t e2 = cudaStreamSynchronize(LN.stream);
        if (e == cudaSuccess) e = e2;
        for (Lane::Arena &A : LN.arena) {
            if (A.p) cudaFreeHost(A.p);
            if (A.ev) cudaEventDestroy(A.ev);
        }
        if (LN.d2h_stage) cudaFreeHost(LN.d2h_stage);
        if (LN.big_copy) cudaEventDestroy(LN.big_copy);
        for (Lane::KTimer &K : LN.ktimer) {
            for (cudaEvent_t e : K.begin) cudaEventDestroy(e);
            for (cudaEvent_t e : K.end) cudaEventDestroy(e);
        }
        if (LN.own_stream) cudaStreamDestroy(LN.own_stream);
    }
    delete ctx;
    return e == cudaSuccess ? VGICP_OK : VGICP_ERR_CUDA;
}

vgicp_status vgicp_set_lane(vgicp_ctx *ctx, int32_t lane, void *cuda_stream)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (lane < 0 || lane >= kMaxLanes) return fail(ctx, VGICP_ERR_INVALID_ARG, "lane must be in [0, %d)", kMaxLanes);
    ctx->lane = lane;
    if (cuda_stream) {
        LN.stream = (cudaStream_t)cuda_stream;
    } else if (!LN.stream) {
        CU(cudaStreamCreateWithFlags(&LN.own_stream, cudaStreamNonBlocking));
        LN.stream = LN.own_stream;
    }
    return VGICP_OK;
}

vgicp_status vgicp_set_options(vgicp_ctx *ctx, const vgicp_options *opt)
{
    if (!ctx || !opt) return VGICP_ERR_INVALID_ARG;
    TRY(check_options(ctx, opt));
    ctx->opt = *opt;
    return VGICP_OK;
}

vgicp_status vgicp_set_stream(vgicp_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    LN.stream = cuda_stream ? (cudaStream_t)cuda_stream : LN.own_stream;
    if (!LN.stream) {
        CU(cudaStreamCreateWithFlags(&LN.own_stream, cudaStreamNonBlocking));
        LN.stream = LN.own_stream;
    }
    return VGICP_OK;
}

vgicp_status vgicp_synchronize(vgicp_ctx *ctx)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    CU(cudaStreamSynchronize(LN.stream));
    return VGICP_OK;
}

// Stage host or device points / covariances in device memory (covs nullable).
namespace {
vgicp_status add_frames_staged(vgicp_ctx *ctx, const float *dp, const float *dc, const int64_t *n, int64_t m,
                               int64_t total, vgicp_frame_t *out);
}

static vgicp_status stage_inputs(vgicp_ctx *ctx, const float *points, const float *covs, int64_t n, int mem_kind,
                                 const float **d_pts, const float **d_cov)
{
    if (mem_kind == VGICP_MEM_DEVICE) {
        *d_pts = points;
        if (d_cov) *d_cov = covs;
        return VGICP_OK;
    }
    const size_t pb = align256((size_t)n * 12), cb = covs ? (size_t)n * 24 : 0;
    TRY(ensure(ctx, LN.ws_stage, pb + cb));
    char *base = (char *)LN.ws_stage.p;
    TRY(h2d(ctx, base, points, (size_t)n * 12));
    if (covs) TRY(h2d(ctx, base + pb, covs, (size_t)n * 24));
    *d_pts = (const float *)base;
    if (d_cov) *d_cov = covs ? (const float *)(base + pb) : nullptr;
    return VGICP_OK;
}

vgicp_status vgicp_add_frame(vgicp_ctx *ctx, const float *points, const float *covs, int64_t n, int mem_kind,
                             vgicp_frame_t *out)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (!out || n < 0 || (n > 0 && (!points || !covs)))
        return fail(ctx, VGICP_ERR_INVALID_ARG, "add_frame: null pointer or negative size");
    if (mem_kind != VGICP_MEM_HOST && mem_kind != VGICP_MEM_DEVICE)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "add_frame: bad mem_kind %d", mem_kind);
    if (n > ((int64_t)1 << 31) - 1) return fail(ctx, VGICP_ERR_INVALID_ARG, "add_frame: n >= 2^31");
    return vgicp_add_frames(ctx, points, covs, &n, 1, mem_kind, out);
}

vgicp_status vgicp_add_frames(vgicp_ctx *ctx, const float *points, const float *covs, const int64_t *n, int64_t m,
                              int mem_kind, vgicp_frame_t *out)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (m < 0 || (m > 0 && (!n || !out)) || m > (1 << 24))
        return fail(ctx, VGICP_ERR_INVALID_ARG, "add_frames: null pointer or bad count");
    if (mem_kind != VGICP_MEM_HOST && mem_kind != VGICP_MEM_DEVICE)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "add_frames: bad mem_kind %d", mem_kind);
    int64_t total = 0;
    for (int64_t u = 0; u < m; ++u) {
        if (n[u] < 0 || n[u] > ((int64_t)1 << 31) - 1)
            return fail(ctx, VGICP_ERR_INVALID_ARG, "add_frames: frame %lld: bad size", (long long)u);
        total += n[u];
    }
    if (total > 0 && (!points || !covs)) return fail(ctx, VGICP_ERR_INVALID_ARG, "add_frames: null pointer");
    if (m == 0) return VGICP_OK;
    const float *dp = nullptr, *dc = nullptr;
    TRY(stage_inputs(ctx, points, covs, total, mem_kind, &dp, &dc));
    return add_frames_staged(ctx, dp, dc, n, m, total, out);
}

}  // extern "C"

namespace {

// Register m frames whose points (total x 3) and covariances (total x 6) are in
// device memory, one frame after another: handles first (all or none), then
// one descriptor scatter and the batched kernels.
vgicp_status add_frames_staged(vgicp_ctx *ctx, const float *dp, const float *dc, const int64_t *n, int64_t m,
                               int64_t total, vgicp_frame_t *out)
{
    std::vector<uint32_t> idx((size_t)m);
    for (int64_t u = 0; u < m; ++u) {
        const vgicp_status st = alloc_frame(ctx, n[u], &idx[u]);
        if (st != VGICP_OK) {
            for (int64_t v = 0; v < u; ++v) vgicp_release(ctx, make_handle(idx[v], ctx->objs[idx[v]].gen));
            return st;
        }
    }
    std::vector<int64_t> off((size_t)m);
    std::vector<int32_t> fidx((size_t)m);
    std::vector<FrameDesc> descs((size_t)m);
    std::vector<WorkItem> items, chunks;
    int64_t o = 0;
    for (int64_t u = 0; u < m; ++u) {
        off[u] = o;
        o += n[u];
        fidx[u] = (int32_t)idx[u];
        descs[u] = ctx->h_frames[idx[u]];
        for (int64_t s0 = 0; s0 < n[u]; s0 += 4096) {
            WorkItem w;
            w.unit = (int32_t)u;
            w.start = s0;
            w.count = (int32_t)std::min<int64_t>(4096, n[u] - s0);
            items.push_back(w);
        }
        for (int c = 0; c < descs[u].nchunks; ++c) {
            WorkItem w;
            w.unit = (int32_t)u;
            w.start = c;
            w.count = 0;
            chunks.push_back(w);
        }
    }
    // one upload: offsets, table indices (twice: as int32 for the kernels and
    // uint32 for the scatter), descriptors, point items, chunk items
    const size_t o_f = align256((size_t)m * 8), o_d = o_f + align256((size_t)m * 4);
    const size_t o_i = o_d + align256((size_t)m * sizeof(FrameDesc));
    const size_t o_c = o_i + align256(items.size() * sizeof(WorkItem));
    const size_t bytes = o_c + chunks.size() * sizeof(WorkItem);
    std::vector<char> host(bytes);
    std::memcpy(host.data(), off.data(), (size_t)m * 8);
    std::memcpy(host.data() + o_f, fidx.data(), (size_t)m * 4);
    std::memcpy(host.data() + o_d, descs.data(), (size_t)m * sizeof(FrameDesc));
    if (!items.empty()) std::memcpy(host.data() + o_i, items.data(), items.size() * sizeof(WorkItem));
    if (!chunks.empty()) std::memcpy(host.data() + o_c, chunks.data(), chunks.size() * sizeof(WorkItem));
    TRY(upload(ctx, LN.ws_descs, host.data(), host.size()));
    char *d = (char *)LN.ws_descs.p;
    bool ordered = false;
    for (int64_t u = 0; u < m; ++u) ordered = ordered || descs[u].perm != nullptr;
    const bool tiles_only = ctx->opt.frame_order == 2;
    if (ordered && !tiles_only) TRY(ensure(ctx, LN.ws_order, (size_t)total * 16));
    launch_frames_register(dp, dc, (const int64_t *)d, (const int32_t *)(d + o_f), (int)m,
                           (const WorkItem *)(d + o_i), (int)items.size(), (const WorkItem *)(d + o_c),
                           (int)chunks.size(), (const uint32_t *)(d + o_f), (const FrameDesc *)(d + o_d),
                           ctx->d_frames, ordered && !tiles_only ? (uint32_t *)LN.ws_order.p : nullptr, total,
                           ctx->num_sms, ordered ? (tiles_only ? 2 : 1) : 0, LN.stream);
    ctx->launches += 2 + (!items.empty()) * (ordered ? 3 : 1) + !chunks.empty();
    CHECK_LAUNCH();
    for (int64_t u = 0; u < m; ++u) out[u] = make_handle(idx[u], ctx->objs[idx[u]].gen);
    return VGICP_OK;
}

}  // namespace

extern "C" {

vgicp_status vgicp_frame_size(vgicp_ctx *ctx, vgicp_frame_t frame, int64_t *n)
{
    if (!ctx || !n) return VGICP_ERR_INVALID_ARG;
    Obj *o = lookup(ctx, frame, Obj::FRAME);
    if (!o) return fail(ctx, VGICP_ERR_NOT_FOUND, "frame handle %lld not found", (long long)frame);
    *n = o->n;
    return VGICP_OK;
}

vgicp_status vgicp_build_voxelmaps(vgicp_ctx *ctx, const vgicp_frame_t *frames, int64_t n, double resolution,
                                   vgicp_map_t *maps)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!frames || !maps))) return fail(ctx, VGICP_ERR_INVALID_ARG, "build_voxelmaps: bad arguments");
    if (!valid_res(resolution)) return fail(ctx, VGICP_ERR_INVALID_ARG, "resolution must be finite and > 0");
    std::vector<uint32_t> fidx(n), midx(n);
    for (int64_t i = 0; i < n; ++i) {
        if (!lookup(ctx, frames[i], Obj::FRAME, &fidx[i]))
            return fail(ctx, VGICP_ERR_NOT_FOUND, "frame handle %lld not found", (long long)frames[i]);
        if (maps[i] >= 0 && !lookup(ctx, maps[i], Obj::MAP, &midx[i]))
            return fail(ctx, VGICP_ERR_NOT_FOUND, "map handle %lld not found", (long long)maps[i]);
    }
    std::vector<uint32_t> upd_idx;
    std::vector<MapDesc> upd;
    for (int64_t i = 0; i < n; ++i) {
        if (maps[i] < 0) {
            TRY(new_obj(ctx, Obj::MAP, &midx[i]));
            maps[i] = make_handle(midx[i], ctx->objs[midx[i]].gen);
        }
        bool changed = false;
        TRY(prepare_map(ctx, midx[i], ctx->objs[fidx[i]].n, resolution, &changed));
        if (changed) {
            upd_idx.push_back(midx[i]);
            upd.push_back(ctx->h_maps[midx[i]]);
        }
    }
    if (n == 0) return VGICP_OK;
    if (!upd.empty()) {
        // one upload and one scatter for every descriptor that changed
        const size_t o_d = align256(upd_idx.size() * 4);
        std::vector<char> host(o_d + upd.size() * sizeof(MapDesc));
        std::memcpy(host.data(), upd_idx.data(), upd_idx.size() * 4);
        std::memcpy(host.data() + o_d, upd.data(), upd.size() * sizeof(MapDesc));
        TRY(upload(ctx, LN.ws_descs, host.data(), host.size()));
        launch_scatter_map_descs((const uint32_t *)LN.ws_descs.p, (const MapDesc *)((char *)LN.ws_descs.p + o_d),
                                 (int)upd.size(), ctx->d_maps, LN.stream);
        ctx->launches += 1;
        CHECK_LAUNCH();
    }
    return run_build(ctx, fidx, midx);
}

vgicp_status vgicp_build_voxelmap(vgicp_ctx *ctx, const float *points, const float *covs, int64_t n,
                                  double resolution, int mem_kind, vgicp_map_t *out)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (!out || n < 0 || (n > 0 && (!points || !covs)))
        return fail(ctx, VGICP_ERR_INVALID_ARG, "build_voxelmap: null pointer or negative size");
    if (!valid_res(resolution)) return fail(ctx, VGICP_ERR_INVALID_ARG, "resolution must be finite and > 0");
    vgicp_frame_t fr;
    TRY(vgicp_add_frame(ctx, points, covs, n, mem_kind, &fr));
    vgicp_map_t m = -1;
    vgicp_status s = vgicp_build_voxelmaps(ctx, &fr, 1, resolution, &m);
    vgicp_release(ctx, fr);
    if (s != VGICP_OK) return s;
    *out = m;
    return VGICP_OK;
}

vgicp_status vgicp_voxelmap_size(vgicp_ctx *ctx, vgicp_map_t map, int64_t *n_voxels)
{
    if (!ctx || !n_voxels) return VGICP_ERR_INVALID_ARG;
    Obj *o = lookup(ctx, map, Obj::MAP);
    if (!o) return fail(ctx, VGICP_ERR_NOT_FOUND, "map handle %lld not found", (long long)map);
    return read_nvox(ctx, *o, n_voxels);
}

}  // extern "C"

namespace {

// Host copy of a spatially ordered frame's storage permutation (empty for a
// frame kept in the given order).
vgicp_status frame_perm(vgicp_ctx *ctx, uint32_t fi, std::vector<int32_t> &perm)
{
    perm.clear();
    const FrameDesc &f = ctx->h_frames[fi];
    if (!f.perm || f.n == 0) return VGICP_OK;
    perm.resize((size_t)f.n);
    CU(cudaMemcpyAsync(perm.data(), f.perm, (size_t)f.n * 4, cudaMemcpyDeviceToHost, LN.stream));
    CU(cudaStreamSynchronize(LN.stream));
    return VGICP_OK;
}

// Per-point rows (w values each) from storage order back to the given order.
template <class T>
void unpermute(T *data, int64_t n, int w, const std::vector<int32_t> &perm)
{
    if (perm.empty() || n == 0) return;
    std::vector<T> tmp(data, data + n * w);
    for (int64_t j = 0; j < n; ++j)
        for (int c = 0; c < w; ++c) data[(int64_t)perm[j] * w + c] = tmp[j * w + c];
}

// Host copy of a correspondence record (CorrRecord layout): voxel coordinates
// unpacked to int64 triples (INT64_MIN on every axis where the point has none
// or was never visited) and the states (-1 where never visited).
struct HostRecord {
    int64_t *keys;
    int32_t *state;
};

// One linearisation of a factor set (the body of vgicp_linearize); with rec,
// the recording instantiations of the same kernels also write each point's
// correspondence, copied to rec's host arrays.
vgicp_status linearize_run(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f, const double *poses,
                           int64_t n_poses, double *H, double *b, double *cost, int64_t *inliers, int out_kind,
                           const HostRecord *rec)
{
    std::vector<int32_t> idx;
    TRY(factor_indices(ctx, factors, n_f, poses, n_poses, idx));
    TRY(upload(ctx, LN.ws_poses, poses, (size_t)n_poses * 12));
    TRY(get_plan(ctx, factors, n_f, idx));
    Plan &P = LN.plan;
    CorrRecord crec{};
    std::vector<int64_t> rbase;
    int64_t rtotal = 0;
    if (rec) {
        rbase.resize((size_t)n_f);
        for (int64_t i = 0; i < n_f; ++i) {
            rbase[i] = rtotal;
            rtotal += ctx->objs[idx[4 * i + 1]].n;
        }
        const size_t o_state = align256((size_t)rtotal * 8), o_base = o_state + align256((size_t)rtotal * 4);
        TRY(ensure(ctx, LN.ws_rec, o_base + (size_t)n_f * 8));
        char *base = (char *)LN.ws_rec.p;
        crec.key = (uint64_t *)base;
        crec.state = (int32_t *)(base + o_state);
        crec.base = (const int64_t *)(base + o_base);
        CU(cudaMemsetAsync(base, 0xff, o_base, LN.stream));   // kEmptyKey, state -1: not visited
        CU(cudaMemcpyAsync(base + o_base, rbase.data(), (size_t)n_f * 8, cudaMemcpyHostToDevice, LN.stream));
    }
    TRY(ensure(ctx, LN.ws_params, (size_t)n_f * sizeof(PoseParam)));
    PoseParam *d_params = (PoseParam *)LN.ws_params.p;
    launch_prepare_factors((const int32_t *)P.idx.p, (int)n_f, (const double *)LN.ws_poses.p, ctx->d_maps,
                           ctx->d_frames, lin_cull(ctx->opt), d_params, LN.stream);
    ctx->launches += 1;
    CHECK_LAUNCH();
    // outputs: caller's device buffers, or a device workspace copied back to the host
    double *dH = H, *db = b, *dc = cost;
    int64_t *di = inliers;
    const size_t out_bytes = (size_t)n_f * (144 + 12 + 1) * 8 + (size_t)n_f * 8;
    if (out_kind == VGICP_MEM_HOST) {
        TRY(ensure(ctx, LN.ws_out, out_bytes));
        dH = (double *)LN.ws_out.p;
        db = dH + n_f * 144;
        dc = db + n_f * 12;
        di = (int64_t *)(dc + n_f);
    }
    if (ctx->opt.precision == VGICP_PREC_F64) {
        const int blk = linearize_f64_block();
        int max_grid = ctx->num_sms * 16;
        TRY(ensure(ctx, LN.ws_f64, (size_t)max_grid * 92 * 8));
        TRY(ensure(ctx, LN.ws_ticket, 4));
        CU(cudaMemsetAsync(LN.ws_ticket.p, 0, 4, LN.stream));
        for (int64_t i = 0; i < n_f; ++i) {
            const int64_t n = ctx->objs[idx[4 * i + 1]].n;
            int grid = (int)std::min<int64_t>(max_grid, std::max<int64_t>(1, (n + blk - 1) / blk));
            launch_linearize_f64(d_params + i, ctx->d_maps, ctx->d_frames, n, (double *)LN.ws_f64.p,
                                 (unsigned int *)LN.ws_ticket.p, dH + 144 * i, db + 12 * i, dc + i,
                                 di ? di + i : nullptr, grid, neighbor_count(ctx->opt), ctx->opt.count_weighted,
                                 LN.stream, rec ? crec.key + rbase[i] : nullptr,
                                 rec ? crec.state + rbase[i] : nullptr);
        }
        ctx->launches += n_f;
        CHECK_LAUNCH();
    } else {
        TRY(ensure(ctx, LN.ws_partials, (size_t)std::max(1, P.n_items) * 28 * 8));
        TRY(ensure(ctx, LN.ws_inl, (size_t)std::max(1, P.n_items) * 8));
        TRY(ensure(ctx, LN.ws_fetch, 16));
        if (uses_img(ctx->opt)) TRY(ensure_images(ctx, idx, n_f));
        const int kt = ktimer_begin(ctx, VGICP_KERNEL_LINEARIZE);
        if (uses_img(ctx->opt))
            launch_linearize_img(d_params, ctx->d_maps, ctx->d_frames, (const WorkItem *)P.items.p,
                                 (const int4 *)P.units.p, P.n_units, (double *)LN.ws_partials.p,
                                 (int64_t *)LN.ws_inl.p, (int *)LN.ws_fetch.p, ctx->num_sms,
                                 ctx->opt.precision == VGICP_PREC_F32_COMP, LN.stream, crec);
        else
            launch_linearize_f32(d_params, ctx->d_maps, ctx->d_frames, (const WorkItem *)P.items.p, P.n_items,
                                 (double *)LN.ws_partials.p, (int64_t *)LN.ws_inl.p, (int *)LN.ws_fetch.p,
                                 ctx->opt.linearize_variant, ctx->opt.blocks_per_sm, ctx->num_sms,
                                 ctx->opt.precision == VGICP_PREC_F32_COMP, neighbor_count(ctx->opt),
                                 ctx->opt.count_weighted, LN.stream, crec);
        ktimer_end(ctx, VGICP_KERNEL_LINEARIZE, kt);
        launch_reduce_finalize(d_params, (const int32_t *)P.item_range.p, (int)n_f, (const double *)LN.ws_partials.p,
                               (const int64_t *)LN.ws_inl.p, dH, db, dc, di, LN.stream);
        ctx->launches += (P.n_items > 0) + 1;
        CHECK_LAUNCH();
    }
    if (out_kind == VGICP_MEM_HOST) {
        void *const dst[4] = {H, b, cost, inliers};
        const size_t nb[4] = {(size_t)n_f * 144 * 8, (size_t)n_f * 12 * 8, (size_t)n_f * 8, (size_t)n_f * 8};
        TRY(d2h_pieces(ctx, dH, dst, nb, 4));
    }
    if (rec && rtotal > 0) {
        std::vector<uint64_t> k((size_t)rtotal);
        CU(cudaMemcpyAsync(k.data(), crec.key, (size_t)rtotal * 8, cudaMemcpyDeviceToHost, LN.stream));
        CU(cudaMemcpyAsync(rec->state, crec.state, (size_t)rtotal * 4, cudaMemcpyDeviceToHost, LN.stream));
        CU(cudaStreamSynchronize(LN.stream));
        for (int64_t j = 0; j < rtotal; ++j) {
            const uint64_t key = k[j];
            for (int a = 0; a < 3; ++a)
                rec->keys[3 * j + a] =
                    key == kEmptyKey ? INT64_MIN
                                     : (int64_t)((key >> (42 - 21 * a)) & 0x1FFFFFull) - (int64_t)kKeyOffset;
        }
        // each factor's points back in its source's given order
        std::vector<int32_t> perm;
        int32_t have = -1;
        for (int64_t i = 0; i < n_f; ++i) {
            const uint32_t fi = (uint32_t)idx[4 * i + 1];
            if ((int32_t)fi != have) {
                TRY(frame_perm(ctx, fi, perm));
                have = (int32_t)fi;
            }
            const int64_t n = ctx->objs[fi].n;
            unpermute(rec->keys + 3 * rbase[i], n, 3, perm);
            unpermute(rec->state + rbase[i], n, 1, perm);
        }
    }
    return VGICP_OK;
}

}  // namespace

extern "C" {

vgicp_status vgicp_linearize(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f, const double *poses,
                             int64_t n_poses, double *H, double *b, double *cost, int64_t *inliers, int out_kind)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (n_f < 0 || n_poses < 0 || (n_f > 0 && (!factors || !H || !b || !cost)) || (n_poses > 0 && !poses))
        return fail(ctx, VGICP_ERR_INVALID_ARG, "linearize: null pointer or negative size");
    if (out_kind != VGICP_MEM_HOST && out_kind != VGICP_MEM_DEVICE)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "linearize: bad out_kind %d", out_kind);
    if (n_f == 0) return VGICP_OK;
    return linearize_run(ctx, factors, n_f, poses, n_poses, H, b, cost, inliers, out_kind, nullptr);
}

vgicp_status vgicp_linearize_correspondences(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f,
                                             const double *poses, int64_t n_poses, double *H, double *b,
                                             double *cost, int64_t *inliers, int64_t *keys, int32_t *state)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (n_f < 0 || n_poses < 0 || (n_f > 0 && (!factors || !keys || !state)) || (n_poses > 0 && !poses))
        return fail(ctx, VGICP_ERR_INVALID_ARG, "linearize_correspondences: null pointer or negative size");
    if (n_f == 0) return VGICP_OK;
    std::vector<double> tmp;
    if (!H || !b || !cost) tmp.resize((size_t)n_f * 157);
    double *h = H ? H : tmp.data(), *bb = b ? b : tmp.data() + n_f * 144, *c = cost ? cost : tmp.data() + n_f * 156;
    const HostRecord rec{keys, state};
    return linearize_run(ctx, factors, n_f, poses, n_poses, h, bb, c, inliers, VGICP_MEM_HOST, &rec);
}

}  // extern "C"

// ---------------------------------------------------------------- plans --
//
// One Gauss-Newton iteration of a fixed factor set as a CUDA graph: the pose
// upload, the per-factor pose preparation, the persistent linearisation launch
// and the fixed-order per-factor reduction, instantiated once and relaunched
// with new poses every iteration.  The graph holds plan-owned buffers only and
// reads descriptor tables at run time, so voxelmaps rebuilt in place between
// iterations are seen; a change of the tables' addresses, of a factor's
// handles or of the kernel options makes the next run capture it again.

struct vgicp_plan {
    std::vector<vgicp_factor> factors;
    std::vector<int32_t> idx;
    std::vector<int64_t> frame_n;
    int64_t n_f = 0, n_poses = 0;
    int n_items = 0;
    Buf d_idx, d_items, d_range, d_poses, d_params, d_partials, d_inl, d_out, d_fetch, d_units;
    int n_units = 0;
    double *h_poses = nullptr;           // pinned staging read by the graph's upload node
    cudaStream_t cap = nullptr;          // capture stream (nothing runs on it)
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    bool in_flight = false;
    // what the graph was captured with
    MapDesc *maps = nullptr;
    FrameDesc *frames = nullptr;
    int chunk = 0, variant = -1, bps = -1, cull = -1, prec = -1, nb = -1, weighted = -1;
    int64_t runs = 0, captures = 0;
};

namespace {

// Resolve the plan's handles; rebuild its work list and graph when anything
// they depend on has changed since the last capture.
vgicp_status plan_refresh(vgicp_ctx *ctx, vgicp_plan *P)
{
    const int64_t n_f = P->n_f;
    std::vector<int32_t> idx((size_t)n_f * 4);
    std::vector<int64_t> fn((size_t)n_f);
    for (int64_t i = 0; i < n_f; ++i) {
        uint32_t mi, fi;
        if (!lookup(ctx, P->factors[i].target, Obj::MAP, &mi))
            return fail(ctx, VGICP_ERR_NOT_FOUND, "plan factor %lld: map handle %lld not found", (long long)i,
                        (long long)P->factors[i].target);
        if (!lookup(ctx, P->factors[i].source, Obj::FRAME, &fi))
            return fail(ctx, VGICP_ERR_NOT_FOUND, "plan factor %lld: frame handle %lld not found", (long long)i,
                        (long long)P->factors[i].source);
        idx[4 * i + 0] = (int32_t)mi;
        idx[4 * i + 1] = (int32_t)fi;
        idx[4 * i + 2] = P->factors[i].target_pose;
        idx[4 * i + 3] = P->factors[i].source_pose;
        fn[i] = ctx->objs[fi].n;
    }
    if (uses_img(ctx->opt)) TRY(ensure_images(ctx, idx, n_f));
    const int chunk = default_chunk(ctx->opt);
    const bool same_work = chunk == P->chunk && idx == P->idx && fn == P->frame_n;
    if (same_work && P->exec && P->maps == ctx->d_maps && P->frames == ctx->d_frames &&
        P->variant == ctx->opt.linearize_variant && P->bps == ctx->opt.blocks_per_sm &&
        P->cull == ctx->opt.linearize_cull && P->prec == ctx->opt.precision && P->nb == neighbor_count(ctx->opt) &&
        P->weighted == ctx->opt.count_weighted)
        return VGICP_OK;
    if (P->in_flight) {
        CU(cudaEventSynchronize(P->done));
        P->in_flight = false;
    }
    if (!same_work) {
        std::vector<WorkItem> items;
        std::vector<int32_t> range;
        build_items(idx, fn, chunk, items, range);
        std::vector<int4> units;
        build_units(idx, items, units);
        TRY(upload(ctx, P->d_units, units.data(), units.size()));
        P->n_units = (int)units.size();
        TRY(upload(ctx, P->d_idx, idx.data(), idx.size()));
        TRY(upload(ctx, P->d_items, items.data(), items.size()));
        TRY(upload(ctx, P->d_range, range.data(), range.size()));
        TRY(ensure(ctx, P->d_partials, std::max<size_t>(1, items.size()) * 28 * 8));
        TRY(ensure(ctx, P->d_inl, std::max<size_t>(1, items.size()) * 8));
        CU(cudaStreamSynchronize(LN.stream));   // buffers ready before the graph can run on any stream
        P->idx = idx;
        P->frame_n = fn;
        P->chunk = chunk;
        P->n_items = (int)items.size();
    }
    if (P->exec) {
        cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
    }
    PoseParam *params = (PoseParam *)P->d_params.p;
    double *H = (double *)P->d_out.p, *b = H + n_f * 144, *c = b + n_f * 12;
    int64_t *inl = (int64_t *)(c + n_f);
    CU(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal));
    cudaMemcpyAsync(P->d_poses.p, P->h_poses, (size_t)P->n_poses * 12 * 8, cudaMemcpyHostToDevice, P->cap);
    launch_prepare_factors((const int32_t *)P->d_idx.p, (int)n_f, (const double *)P->d_poses.p, ctx->d_maps,
                           ctx->d_frames, lin_cull(ctx->opt), params, P->cap);
    if (uses_img(ctx->opt))
        launch_linearize_img(params, ctx->d_maps, ctx->d_frames, (const WorkItem *)P->d_items.p,
                             (const int4 *)P->d_units.p, P->n_units, (double *)P->d_partials.p,
                             (int64_t *)P->d_inl.p, (int *)P->d_fetch.p, ctx->num_sms,
                             ctx->opt.precision == VGICP_PREC_F32_COMP, P->cap);
    else
        launch_linearize_f32(params, ctx->d_maps, ctx->d_frames, (const WorkItem *)P->d_items.p, P->n_items,
                             (double *)P->d_partials.p, (int64_t *)P->d_inl.p, (int *)P->d_fetch.p,
                             ctx->opt.linearize_variant, ctx->opt.blocks_per_sm, ctx->num_sms,
                             ctx->opt.precision == VGICP_PREC_F32_COMP, neighbor_count(ctx->opt),
                             ctx->opt.count_weighted, P->cap);
    launch_reduce_finalize(params, (const int32_t *)P->d_range.p, (int)n_f, (const double *)P->d_partials.p,
                           (const int64_t *)P->d_inl.p, H, b, c, inl, P->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e1 = cudaStreamEndCapture(P->cap, &g);
    const cudaError_t e0 = cudaGetLastError();
    if (e1 != cudaSuccess || e0 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(ctx, VGICP_ERR_CUDA, "plan capture: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e0));
    }
    const cudaError_t e2 = cudaGraphInstantiate(&P->exec, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
        P->exec = nullptr;
        return fail(ctx, VGICP_ERR_CUDA, "plan instantiate: %s", cudaGetErrorString(e2));
    }
    P->maps = ctx->d_maps;
    P->frames = ctx->d_frames;
    P->variant = ctx->opt.linearize_variant;
    P->bps = ctx->opt.blocks_per_sm;
    P->cull = ctx->opt.linearize_cull;
    P->prec = ctx->opt.precision;
    P->nb = neighbor_count(ctx->opt);
    P->weighted = ctx->opt.count_weighted;
    P->captures += 1;
    return VGICP_OK;
}

void plan_free(vgicp_ctx *ctx, vgicp_plan *P)
{
    if (P->in_flight) cudaEventSynchronize(P->done);
    if (P->exec) cudaGraphExecDestroy(P->exec);
    Buf *bufs[] = {&P->d_idx, &P->d_items, &P->d_range, &P->d_poses, &P->d_params, &P->d_partials, &P->d_inl,
                   &P->d_out, &P->d_fetch, &P->d_units};
    for (Buf *b : bufs) free_buf(ctx, *b);
    if (P->h_poses) cudaFreeHost(P->h_poses);
    if (P->done) cudaEventDestroy(P->done);
    if (P->cap) cudaStreamDestroy(P->cap);
    delete P;
}

}  // namespace

extern "C" {

vgicp_status vgicp_plan_create(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f, int64_t n_poses,
                               vgicp_plan **plan)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (!plan || n_f < 0 || n_poses < 0 || (n_f > 0 && !factors) || n_f > (1 << 30))
        return fail(ctx, VGICP_ERR_INVALID_ARG, "plan_create: null pointer or bad size");
    *plan = nullptr;
    for (int64_t i = 0; i < n_f; ++i)
        if (factors[i].target_pose < 0 || factors[i].target_pose >= n_poses || factors[i].source_pose < 0 ||
            factors[i].source_pose >= n_poses)
            return fail(ctx, VGICP_ERR_INVALID_ARG, "plan factor %lld: pose index out of range", (long long)i);
    vgicp_plan *P = new vgicp_plan();
    P->factors.assign(factors, factors + n_f);
    P->n_f = n_f;
    P->n_poses = n_poses;
    vgicp_status st = VGICP_OK;
    auto cu = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && st == VGICP_OK)
            st = fail(ctx, e == cudaErrorMemoryAllocation ? VGICP_ERR_OOM : VGICP_ERR_CUDA, "plan_create: %s: %s",
                      what, cudaGetErrorString(e));
    };
    cu(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking), "stream");
    cu(cudaEventCreateWithFlags(&P->done, cudaEventDisableTiming), "event");
    cu(cudaMallocHost(&P->h_poses, (size_t)std::max<int64_t>(1, n_poses) * 12 * 8), "pinned poses");
    if (st == VGICP_OK) st = ensure(ctx, P->d_poses, (size_t)std::max<int64_t>(1, n_poses) * 12 * 8);
    if (st == VGICP_OK) st = ensure(ctx, P->d_params, (size_t)std::max<int64_t>(1, n_f) * sizeof(PoseParam));
    if (st == VGICP_OK) st = ensure(ctx, P->d_out, (size_t)std::max<int64_t>(1, n_f) * (144 + 12 + 1 + 1) * 8);
    if (st == VGICP_OK) st = ensure(ctx, P->d_fetch, 16);
    if (st == VGICP_OK && n_f > 0) st = plan_refresh(ctx, P);
    if (st != VGICP_OK) {
        plan_free(ctx, P);
        return st;
    }
    *plan = P;
    return VGICP_OK;
}

vgicp_status vgicp_plan_linearize(vgicp_ctx *ctx, vgicp_plan *P, const double *poses, double *H, double *b,
                                  double *cost, int64_t *inliers, int out_kind)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (!P || (P->n_poses > 0 && !poses) || (P->n_f > 0 && (!H || !b || !cost)))
        return fail(ctx, VGICP_ERR_INVALID_ARG, "plan_linearize: null pointer");
    if (out_kind != VGICP_MEM_HOST && out_kind != VGICP_MEM_DEVICE)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "plan_linearize: bad out_kind %d", out_kind);
    if (P->n_f == 0) return VGICP_OK;
    for (int64_t i = 0; i < P->n_poses * 12; ++i)
        if (!std::isfinite(poses[i])) return fail(ctx, VGICP_ERR_INVALID_ARG, "plan_linearize: non-finite pose");
    if (ctx->opt.precision == VGICP_PREC_F64)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "plan_linearize: plans run the batched float32 path");
    TRY(plan_refresh(ctx, P));
    if (P->in_flight) CU(cudaEventSynchronize(P->done));   // the previous run has read the staging buffer
    std::memcpy(P->h_poses, poses, (size_t)P->n_poses * 12 * 8);
    CU(cudaGraphLaunch(P->exec, LN.stream));
    CU(cudaEventRecord(P->done, LN.stream));
    P->in_flight = true;
    P->runs += 1;
    ctx->launches += 2 + (P->n_items > 0);
    const int64_t n_f = P->n_f;
    const double *dH = (const double *)P->d_out.p, *db = dH + n_f * 144, *dc = db + n_f * 12;
    const int64_t *di = (const int64_t *)(dc + n_f);
    const cudaMemcpyKind k = out_kind == VGICP_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    CU(cudaMemcpyAsync(H, dH, (size_t)n_f * 144 * 8, k, LN.stream));
    CU(cudaMemcpyAsync(b, db, (size_t)n_f * 12 * 8, k, LN.stream));
    CU(cudaMemcpyAsync(cost, dc, (size_t)n_f * 8, k, LN.stream));
    if (inliers) CU(cudaMemcpyAsync(inliers, di, (size_t)n_f * 8, k, LN.stream));
    if (out_kind == VGICP_MEM_HOST) CU(cudaStreamSynchronize(LN.stream));
    return VGICP_OK;
}

vgicp_status vgicp_plan_info(vgicp_ctx *ctx, const vgicp_plan *P, int64_t *runs, int64_t *captures)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (!P) return fail(ctx, VGICP_ERR_INVALID_ARG, "plan_info: null plan");
    if (runs) *runs = P->runs;
    if (captures) *captures = P->captures;
    return VGICP_OK;
}

vgicp_status vgicp_plan_destroy(vgicp_ctx *ctx, vgicp_plan *P)
{
    if (!ctx || !P) return VGICP_ERR_INVALID_ARG;
    plan_free(ctx, P);
    return VGICP_OK;
}

}  // extern "C"

extern "C" {

vgicp_status vgicp_evaluate(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f, const double *poses,
                            int64_t n_poses, double *cost, int64_t *inliers, int out_kind)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (n_f < 0 || n_poses < 0 || (n_f > 0 && (!factors || !cost)) || (n_poses > 0 && !poses))
        return fail(ctx, VGICP_ERR_INVALID_ARG, "evaluate: null pointer or negative size");
    if (out_kind != VGICP_MEM_HOST && out_kind != VGICP_MEM_DEVICE)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "evaluate: bad out_kind %d", out_kind);
    if (n_f == 0) return VGICP_OK;
    std::vector<int32_t> idx;
    TRY(factor_indices(ctx, factors, n_f, poses, n_poses, idx));
    TRY(upload(ctx, LN.ws_poses, poses, (size_t)n_poses * 12));
    TRY(get_plan(ctx, factors, n_f, idx));
    Plan &P = LN.plan;
    TRY(ensure(ctx, LN.ws_params, (size_t)n_f * sizeof(PoseParam)));
    PoseParam *d_params = (PoseParam *)LN.ws_params.p;
    launch_prepare_factors((const int32_t *)P.idx.p, (int)n_f, (const double *)LN.ws_poses.p, ctx->d_maps,
                           ctx->d_frames, lin_cull(ctx->opt), d_params, LN.stream);
    double *dc = cost;
    int64_t *di = inliers;
    if (out_kind == VGICP_MEM_HOST) {
        TRY(ensure(ctx, LN.ws_out, (size_t)n_f * 16));
        dc = (double *)LN.ws_out.p;
        di = (int64_t *)(dc + n_f);
    }
    TRY(ensure(ctx, LN.ws_partials, (size_t)std::max(1, P.n_items) * 8));
    TRY(ensure(ctx, LN.ws_inl, (size_t)std::max(1, P.n_items) * 8));
    TRY(ensure(ctx, LN.ws_fetch, 16));
    launch_cost_f32(d_params, ctx->d_maps, ctx->d_frames, (const WorkItem *)P.items.p, P.n_items,
                    (double *)LN.ws_partials.p, (int64_t *)LN.ws_inl.p, (int *)LN.ws_fetch.p,
                    ctx->opt.linearize_variant, ctx->opt.blocks_per_sm, ctx->num_sms,
                    ctx->opt.precision == VGICP_PREC_F32_COMP, neighbor_count(ctx->opt), ctx->opt.count_weighted,
                    LN.stream);
    launch_reduce_cost((const int32_t *)P.item_range.p, (int)n_f, (const double *)LN.ws_partials.p,
                       (const int64_t *)LN.ws_inl.p, dc, di, LN.stream);
    ctx->launches += 2 + (P.n_items > 0);
    CHECK_LAUNCH();
    if (out_kind == VGICP_MEM_HOST) {
        void *const dst[2] = {cost, inliers};
        const size_t nb[2] = {(size_t)n_f * 8, (size_t)n_f * 8};
        TRY(d2h_pieces(ctx, dc, dst, nb, 2));
    }
    return VGICP_OK;
}

vgicp_status vgicp_autotune(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f, const double *poses,
                            int64_t n_poses, int32_t reps, vgicp_options *best, double *best_ms)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (n_f <= 0 || reps < 1 || !factors || !poses)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "autotune: needs factors, poses and reps >= 1");
    const size_t out = (size_t)n_f * (144 + 12 + 1 + 1) * 8;
    TRY(ensure(ctx, LN.ws_tune, out));
    double *H = (double *)LN.ws_tune.p, *b = H + n_f * 144, *c = b + n_f * 12;
    int64_t *inl = (int64_t *)(c + n_f);
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    const vgicp_options keep = ctx->opt;
    vgicp_options win = keep;
    float win_ms = 1e30f;
    static const int chunks[] = {1024, 2048, 4096, 8192};
    vgicp_status st = VGICP_OK;
    for (int variant = 0; variant <= 6 && st == VGICP_OK; ++variant)
        for (int ci = 0; ci < 4 && st == VGICP_OK; ++ci) {
            ctx->opt = keep;
            if (keep.precision == VGICP_PREC_F64) ctx->opt.precision = VGICP_PREC_F32;
            ctx->opt.linearize_variant = variant;
            ctx->opt.chunk_points = chunks[ci];
            ctx->opt.blocks_per_sm = 0;
            st = vgicp_linearize(ctx, factors, n_f, poses, n_poses, H, b, c, inl, VGICP_MEM_DEVICE);
            if (st != VGICP_OK) break;
            cudaEventRecord(e0, LN.stream);
            for (int r = 0; r < reps && st == VGICP_OK; ++r)
                st = vgicp_linearize(ctx, factors, n_f, poses, n_poses, H, b, c, inl, VGICP_MEM_DEVICE);
            cudaEventRecord(e1, LN.stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) { st = fail(ctx, VGICP_ERR_CUDA, "autotune: event"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)reps;
            if (ms < win_ms) {
                win_ms = ms;
                win = ctx->opt;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != VGICP_OK) {
        ctx->opt = keep;
        return st;
    }
    ctx->opt = win;
    if (best) *best = win;
    if (best_ms) *best_ms = win_ms;
    return VGICP_OK;
}

vgicp_status vgicp_overlap(vgicp_ctx *ctx, vgicp_frame_t source, vgicp_map_t target, const double *T, double *fraction,
                           int64_t *count)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (!T || !fraction) return fail(ctx, VGICP_ERR_INVALID_ARG, "overlap: null pointer");
    uint32_t fi, mi;
    Obj *fo = lookup(ctx, source, Obj::FRAME, &fi);
    if (!fo) return fail(ctx, VGICP_ERR_NOT_FOUND, "frame handle %lld not found", (long long)source);
    if (!lookup(ctx, target, Obj::MAP, &mi))
        return fail(ctx, VGICP_ERR_NOT_FOUND, "map handle %lld not found", (long long)target);
    if (!finite_pose(T)) return fail(ctx, VGICP_ERR_INVALID_ARG, "overlap: non-finite pose");
    const int64_t n = fo->n;
    if (n == 0) return fail(ctx, VGICP_ERR_EMPTY, "overlap of an empty source is undefined (Eq. 8)");
    std::vector<WorkItem> items;
    for (int64_t s = 0; s < n; s += 4096) {
        WorkItem w;
        w.unit = 0;
        w.start = s;
        w.count = (int32_t)std::min<int64_t>(4096, n - s);
        items.push_back(w);
    }
    TRY(upload(ctx, LN.ws_poses, T, 12));
    TRY(ensure(ctx, LN.ws_pairs, sizeof(PoseParam)));
    LN.last_matrix_pairs = 0;
    launch_prepare_given((const double *)LN.ws_poses.p, (int)mi, (int)fi, ctx->d_maps, ctx->d_frames,
                         ov_cull(ctx->opt), (PoseParam *)LN.ws_pairs.p, LN.stream);
    ctx->launches += 1;
    TRY(upload(ctx, LN.ws_chunks, items.data(), items.size()));
    TRY(ensure(ctx, LN.ws_counts, 8));
    CU(cudaMemsetAsync(LN.ws_counts.p, 0, 8, LN.stream));
    const int grid = std::max(1, std::min((int)items.size(), ctx->num_sms * 8));
    launch_overlap((const PoseParam *)LN.ws_pairs.p, ctx->d_maps, ctx->d_frames, (const WorkItem *)LN.ws_chunks.p,
                   (int)items.size(), (unsigned long long *)LN.ws_counts.p, grid, LN.stream);
    ctx->launches += 1;
    CHECK_LAUNCH();
    unsigned long long c = 0;
    {
        void *const dst[1] = {&c};
        const size_t nb[1] = {8};
        TRY(d2h_pieces(ctx, LN.ws_counts.p, dst, nb, 1));
    }
    if (count) *count = (int64_t)c;
    *fraction = (double)c / (double)n;
    return VGICP_OK;
}

vgicp_status vgicp_overlap_pairs(vgicp_ctx *ctx, const vgicp_frame_t *sources, const vgicp_map_t *targets,
                                 int64_t n, const double *T, int64_t *counts, int out_kind)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!sources || !targets || !T || !counts)))
        return fail(ctx, VGICP_ERR_INVALID_ARG, "overlap_pairs: null pointer or negative size");
    if (out_kind != VGICP_MEM_HOST && out_kind != VGICP_MEM_DEVICE)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "overlap_pairs: bad out_kind %d", out_kind);
    if (n == 0) return VGICP_OK;
    if (n > (1 << 30)) return fail(ctx, VGICP_ERR_INVALID_ARG, "overlap_pairs: too many pairs");
    std::vector<int32_t> idx((size_t)n * 2);
    std::vector<WorkItem> items;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t fi, mi;
        Obj *fo = lookup(ctx, sources[i], Obj::FRAME, &fi);
        if (!fo) return fail(ctx, VGICP_ERR_NOT_FOUND, "pair %lld: frame handle not found", (long long)i);
        if (!lookup(ctx, targets[i], Obj::MAP, &mi))
            return fail(ctx, VGICP_ERR_NOT_FOUND, "pair %lld: map handle not found", (long long)i);
        if (!finite_pose(T + 12 * i)) return fail(ctx, VGICP_ERR_INVALID_ARG, "pair %lld: non-finite pose", (long long)i);
        idx[i] = (int32_t)mi;
        idx[n + i] = (int32_t)fi;
        for (int64_t s = 0; s < fo->n; s += 4096) {
            WorkItem w;
            w.unit = (int32_t)i;
            w.start = s;
            w.count = (int32_t)std::min<int64_t>(4096, fo->n - s);
            items.push_back(w);
        }
    }
    TRY(upload(ctx, LN.ws_poses, T, (size_t)n * 12));
    TRY(upload(ctx, LN.ws_fidx, idx.data(), idx.size()));
    TRY(upload(ctx, LN.ws_chunks, items.data(), items.size()));
    TRY(ensure(ctx, LN.ws_pairs, (size_t)n * sizeof(PoseParam)));
    LN.last_matrix_pairs = 0;
    const int32_t *d_idx = (const int32_t *)LN.ws_fidx.p;
    launch_prepare_list((const double *)LN.ws_poses.p, d_idx, d_idx + n, (int)n, ctx->d_maps, ctx->d_frames,
                        ov_cull(ctx->opt), (PoseParam *)LN.ws_pairs.p, LN.stream);
    unsigned long long *dc = (unsigned long long *)counts;
    if (out_kind == VGICP_MEM_HOST) {
        TRY(ensure(ctx, LN.ws_counts, (size_t)n * 8));
        dc = (unsigned long long *)LN.ws_counts.p;
    }
    CU(cudaMemsetAsync(dc, 0, (size_t)n * 8, LN.stream));
    const int grid = std::max(1, std::min((int)items.size(), ctx->num_sms * 8));
    launch_overlap((const PoseParam *)LN.ws_pairs.p, ctx->d_maps, ctx->d_frames, (const WorkItem *)LN.ws_chunks.p,
                   (int)items.size(), dc, grid, LN.stream);
    ctx->launches += 1 + !items.empty();
    CHECK_LAUNCH();
    if (out_kind == VGICP_MEM_HOST) {
        void *const dst[1] = {counts};
        const size_t nb[1] = {(size_t)n * 8};
        TRY(d2h_pieces(ctx, dc, dst, nb, 1));
    }
    return VGICP_OK;
}

vgicp_status vgicp_overlap_matrix(vgicp_ctx *ctx, const vgicp_frame_t *sources, int64_t n_src,
                                  const vgicp_map_t *targets, int64_t n_tgt, const double *poses_src,
                                  const double *poses_tgt, int64_t *counts, int out_kind)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (n_src < 0 || n_tgt < 0 || (n_src > 0 && (!sources || !poses_src)) || (n_tgt > 0 && (!targets || !poses_tgt)) ||
        (n_src * n_tgt > 0 && !counts))
        return fail(ctx, VGICP_ERR_INVALID_ARG, "overlap_matrix: null pointer or negative size");
    if (out_kind != VGICP_MEM_HOST && out_kind != VGICP_MEM_DEVICE)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "overlap_matrix: bad out_kind %d", out_kind);
    const int64_t n_pairs = n_src * n_tgt;
    if (n_pairs == 0) return VGICP_OK;
    if (n_pairs > (int64_t)1 << 30) return fail(ctx, VGICP_ERR_INVALID_ARG, "overlap_matrix: too many pairs");
    std::vector<int32_t> fidx(n_src), midx(n_tgt);
    std::vector<int64_t> nsrc(n_src);
    for (int64_t i = 0; i < n_src; ++i) {
        uint32_t k;
        Obj *o = lookup(ctx, sources[i], Obj::FRAME, &k);
        if (!o) return fail(ctx, VGICP_ERR_NOT_FOUND, "frame handle %lld not found", (long long)sources[i]);
        fidx[i] = (int32_t)k;
        nsrc[i] = o->n;
    }
    for (int64_t i = 0; i < n_tgt; ++i) {
        uint32_t k;
        Obj *o = lookup(ctx, targets[i], Obj::MAP, &k);
        if (!o) return fail(ctx, VGICP_ERR_NOT_FOUND, "map handle %lld not found", (long long)targets[i]);
        midx[i] = (int32_t)k;
    }
    for (int64_t i = 0; i < n_src * 12; ++i)
        if (!std::isfinite(poses_src[i])) return fail(ctx, VGICP_ERR_INVALID_ARG, "overlap_matrix: non-finite pose");
    for (int64_t i = 0; i < n_tgt * 12; ++i)
        if (!std::isfinite(poses_tgt[i])) return fail(ctx, VGICP_ERR_INVALID_ARG, "overlap_matrix: non-finite pose");
    TRY(upload(ctx, LN.ws_poses, poses_src, (size_t)n_src * 12));
    TRY(ensure(ctx, LN.ws_stage, (size_t)n_tgt * 12 * 8));
    TRY(h2d(ctx, LN.ws_stage.p, poses_tgt, (size_t)n_tgt * 12 * 8));
    TRY(upload(ctx, LN.ws_fidx, fidx.data(), fidx.size()));
    TRY(upload(ctx, LN.ws_midx, midx.data(), midx.size()));
    TRY(ensure(ctx, LN.ws_pairs, (size_t)n_pairs * sizeof(PoseParam)));
    launch_prepare_pairs((const double *)LN.ws_poses.p, (const double *)LN.ws_stage.p,
                         (const int32_t *)LN.ws_fidx.p, (const int32_t *)LN.ws_midx.p, (int)n_src, (int)n_tgt,
                         ctx->d_maps, ctx->d_frames, ov_cull(ctx->opt), (PoseParam *)LN.ws_pairs.p,
                         LN.stream);
    LN.last_matrix_pairs = n_pairs;
    unsigned long long *dcounts = (unsigned long long *)counts;
    if (out_kind == VGICP_MEM_HOST) {
        TRY(ensure(ctx, LN.ws_counts, (size_t)n_pairs * 8));
        dcounts = (unsigned long long *)LN.ws_counts.p;
    }
    CU(cudaMemsetAsync(dcounts, 0, (size_t)n_pairs * 8, LN.stream));
    TRY(ensure(ctx, LN.ws_items, overlap_matrix_scratch_bytes((int)n_src, (int)n_tgt)));
    const int kt = ktimer_begin(ctx, VGICP_KERNEL_OVERLAP_MATRIX);
    launch_overlap_matrix((const PoseParam *)LN.ws_pairs.p, ctx->d_maps, ctx->d_frames, (int)n_src, (int)n_tgt,
                          dcounts, LN.ws_items.p, ctx->num_sms, LN.stream);
    ktimer_end(ctx, VGICP_KERNEL_OVERLAP_MATRIX, kt);
    ctx->launches += 4;   // pair preparation, item lists, the two matrix kernels
    CHECK_LAUNCH();
    if (out_kind == VGICP_MEM_HOST) {
        void *const dst[1] = {counts};
        const size_t nb[1] = {(size_t)n_pairs * 8};
        TRY(d2h_pieces(ctx, dcounts, dst, nb, 1));
    }
    return VGICP_OK;
}

vgicp_status vgicp_overlap_matrix_work(vgicp_ctx *ctx, int64_t *live_pairs, int64_t *lookups)
{
    if (!ctx || !live_pairs || !lookups) return VGICP_ERR_INVALID_ARG;
    *live_pairs = 0;
    *lookups = 0;
    if (LN.last_matrix_pairs <= 0) return VGICP_OK;
    TRY(ensure(ctx, LN.ws_counter, 16));
    CU(cudaMemsetAsync(LN.ws_counter.p, 0, 16, LN.stream));
    launch_count_live((const PoseParam *)LN.ws_pairs.p, LN.last_matrix_pairs, ctx->d_frames, ctx->d_maps,
                      (unsigned long long *)LN.ws_counter.p, LN.stream);
    ctx->launches += 1;
    CHECK_LAUNCH();
    unsigned long long h[2];
    CU(cudaMemcpyAsync(h, LN.ws_counter.p, 16, cudaMemcpyDeviceToHost, LN.stream));
    CU(cudaStreamSynchronize(LN.stream));
    *live_pairs = (int64_t)h[0];
    *lookups = (int64_t)h[1];
    return VGICP_OK;
}

vgicp_status vgicp_debug_correspondences(vgicp_ctx *ctx, vgicp_frame_t source, vgicp_map_t target, const double *T,
                                         int64_t *keys, int32_t *hit)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (!T) return fail(ctx, VGICP_ERR_INVALID_ARG, "debug_correspondences: null pose");
    uint32_t fi, mi;
    Obj *fo = lookup(ctx, source, Obj::FRAME, &fi);
    if (!fo) return fail(ctx, VGICP_ERR_NOT_FOUND, "frame handle %lld not found", (long long)source);
    if (!lookup(ctx, target, Obj::MAP, &mi))
        return fail(ctx, VGICP_ERR_NOT_FOUND, "map handle %lld not found", (long long)target);
    const int64_t n = fo->n;
    if (n == 0) return VGICP_OK;
    TRY(upload(ctx, LN.ws_poses, T, 12));
    TRY(ensure(ctx, LN.ws_pairs, sizeof(PoseParam)));
    LN.last_matrix_pairs = 0;
    launch_prepare_given((const double *)LN.ws_poses.p, (int)mi, (int)fi, ctx->d_maps, ctx->d_frames, 0,
                         (PoseParam *)LN.ws_pairs.p, LN.stream);
    ctx->launches += 1;
    TRY(ensure(ctx, LN.ws_out, (size_t)n * (24 + 4)));
    int64_t *dk = (int64_t *)LN.ws_out.p;
    int32_t *dh = (int32_t *)(dk + 3 * n);
    launch_correspondences((const PoseParam *)LN.ws_pairs.p, ctx->d_maps, ctx->d_frames, n, dk, dh, LN.stream);
    ctx->launches += 1;
    CHECK_LAUNCH();
    if (keys) CU(cudaMemcpyAsync(keys, dk, (size_t)n * 24, cudaMemcpyDeviceToHost, LN.stream));
    if (hit) CU(cudaMemcpyAsync(hit, dh, (size_t)n * 4, cudaMemcpyDeviceToHost, LN.stream));
    CU(cudaStreamSynchronize(LN.stream));
    std::vector<int32_t> perm;
    TRY(frame_perm(ctx, fi, perm));
    if (keys) unpermute(keys, n, 3, perm);
    if (hit) unpermute(hit, n, 1, perm);
    return VGICP_OK;
}

vgicp_status vgicp_export_voxelmap(vgicp_ctx *ctx, vgicp_map_t map, int64_t *keys, int64_t *counts, double *mu,
                                   double *cov, int64_t *n_voxels)
{
    if (!ctx || !n_voxels) return VGICP_ERR_INVALID_ARG;
    uint32_t mi;
    Obj *o = lookup(ctx, map, Obj::MAP, &mi);
    if (!o) return fail(ctx, VGICP_ERR_NOT_FOUND, "map handle %lld not found", (long long)map);
    int64_t nv;
    TRY(read_nvox(ctx, *o, &nv));
    const int64_t capacity = *n_voxels;
    *n_voxels = nv;
    if (!keys && !counts && !mu && !cov) return VGICP_OK;
    if (capacity < nv) return fail(ctx, VGICP_ERR_INVALID_ARG, "export: capacity %lld < %lld voxels",
                                   (long long)capacity, (long long)nv);
    TRY(ensure(ctx, LN.ws_export_keys, (size_t)std::max<int64_t>(nv, 1) * 8));
    TRY(ensure(ctx, LN.ws_export_rec, (size_t)std::max<int64_t>(nv, 1) * sizeof(VoxelRec)));
    TRY(ensure(ctx, LN.ws_counter, 4));
    CU(cudaMemsetAsync(LN.ws_counter.p, 0, 4, LN.stream));
    launch_export_voxels(ctx->d_maps + mi, o->cap, (uint32_t *)LN.ws_counter.p, (uint64_t *)LN.ws_export_keys.p,
                         (VoxelRec *)LN.ws_export_rec.p, LN.stream);
    ctx->launches += 1;
    CHECK_LAUNCH();
    std::vector<uint64_t> hk(nv);
    std::vector<VoxelRec> hr(nv);
    if (nv) {
        CU(cudaMemcpyAsync(hk.data(), LN.ws_export_keys.p, (size_t)nv * 8, cudaMemcpyDeviceToHost, LN.stream));
        CU(cudaMemcpyAsync(hr.data(), LN.ws_export_rec.p, (size_t)nv * sizeof(VoxelRec), cudaMemcpyDeviceToHost,
                           LN.stream));
    }
    CU(cudaStreamSynchronize(LN.stream));
    std::vector<int64_t> order(nv);
    for (int64_t i = 0; i < nv; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return hk[a] < hk[b]; });
    const double r = o->r;
    for (int64_t j = 0; j < nv; ++j) {
        const uint64_t k = hk[order[j]];
        const VoxelRec &v = hr[order[j]];
        const int64_t kk[3] = {(int64_t)((k >> 42) & 0x1FFFFF) - kKeyOffset, (int64_t)((k >> 21) & 0x1FFFFF) - kKeyOffset,
                               (int64_t)(k & 0x1FFFFF) - kKeyOffset};
        if (keys) for (int a = 0; a < 3; ++a) keys[3 * j + a] = kk[a];
        uint32_t cnt;
        std::memcpy(&cnt, &v.c.y, 4);
        if (counts) counts[j] = cnt;
        if (mu) {
            mu[3 * j + 0] = (double)kk[0] * r + (double)v.a.x;
            mu[3 * j + 1] = (double)kk[1] * r + (double)v.a.y;
            mu[3 * j + 2] = (double)kk[2] * r + (double)v.a.z;
        }
        if (cov) {
            cov[6 * j + 0] = v.a.w; cov[6 * j + 1] = v.b.x; cov[6 * j + 2] = v.b.y;
            cov[6 * j + 3] = v.b.z; cov[6 * j + 4] = v.b.w; cov[6 * j + 5] = v.c.x;
        }
    }
    return VGICP_OK;
}

vgicp_status vgicp_estimate_covariances(vgicp_ctx *ctx, const float *points, int64_t n, int32_t k, double eps,
                                        float *covs_out, int mem_kind)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!points || !covs_out)) || k < 1 || k > 32 || !std::isfinite(eps))
        return fail(ctx, VGICP_ERR_INVALID_ARG, "estimate_covariances: bad arguments");
    if (mem_kind != VGICP_MEM_HOST && mem_kind != VGICP_MEM_DEVICE)
        return fail(ctx, VGICP_ERR_INVALID_ARG, "estimate_covariances: bad mem_kind");
    if (n == 0) return VGICP_OK;
    const float *dp;
    TRY(stage_inputs(ctx, points, nullptr, n, mem_kind, &dp, nullptr));
    float *dc = covs_out;
    if (mem_kind == VGICP_MEM_HOST) {
        TRY(ensure(ctx, LN.ws_out, (size_t)n * 24));
        dc = (float *)LN.ws_out.p;
    }
    TRY(ensure(ctx, LN.ws_knn, knn_scratch_bytes(n)));
    launch_knn_covariances(dp, n, k, eps, 1.0, LN.ws_knn.p, dc, LN.stream);
    ctx->launches += 5;
    CHECK_LAUNCH();
    if (mem_kind == VGICP_MEM_HOST) {
        CU(cudaMemcpyAsync(covs_out, dc, (size_t)n * 24, cudaMemcpyDeviceToHost, LN.stream));
        CU(cudaStreamSynchronize(LN.stream));
    }
    return VGICP_OK;
}

vgicp_status vgicp_release(vgicp_ctx *ctx, int64_t handle)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    uint32_t idx;
    Obj *o = lookup(ctx, handle, Obj::FRAME, &idx);
    if (!o) o = lookup(ctx, handle, Obj::MAP, &idx);
    if (!o) return fail(ctx, VGICP_ERR_NOT_FOUND, "handle %lld not found", (long long)handle);
    if (o->frame_mem) CU(cudaFreeAsync(o->frame_mem, LN.stream));
    if (o->map_mem) CU(cudaFreeAsync(o->map_mem, LN.stream));
    ctx->bytes_in_use -= (int64_t)(o->frame_bytes + o->map_bytes);
    const uint32_t gen = o->gen;
    *o = Obj();
    o->gen = gen;
    if (ctx->idx_ev.size() <= idx) {
        ctx->idx_ev.resize(idx + 1, nullptr);
        ctx->idx_ev_set.resize(idx + 1, 0);
    }
    if (!ctx->idx_ev[idx]) CU(cudaEventCreateWithFlags(&ctx->idx_ev[idx], cudaEventDisableTiming));
    CU(cudaEventRecord(ctx->idx_ev[idx], LN.stream));
    ctx->idx_ev_set[idx] = 1;
    ctx->free_idx.push_back(idx);
    LN.plan.key.clear();   // a cached work list may name this handle
    return VGICP_OK;
}

vgicp_status vgicp_release_many(vgicp_ctx *ctx, const int64_t *handles, int64_t n)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && !handles)) return fail(ctx, VGICP_ERR_INVALID_ARG, "release_many: bad arguments");
    for (int64_t i = 0; i < n; ++i)
        if (!lookup(ctx, handles[i], Obj::FRAME) && !lookup(ctx, handles[i], Obj::MAP))
            return fail(ctx, VGICP_ERR_NOT_FOUND, "release_many: handle %lld not found", (long long)handles[i]);
    for (int64_t i = 0; i < n; ++i) {
        const vgicp_status st = vgicp_release(ctx, handles[i]);
        if (st != VGICP_OK) return st;    // a handle listed twice
    }
    return VGICP_OK;
}

vgicp_status vgicp_memory_estimate(vgicp_ctx *ctx, int64_t n, int32_t is_map, int64_t *bytes)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (!bytes || n < 0) return fail(ctx, VGICP_ERR_INVALID_ARG, "memory_estimate: bad arguments");
    *bytes = is_map ? (int64_t)map_bytes(map_capacity(n))
                    : (int64_t)frame_bytes(n, ctx->opt.frame_order != 0 && n > 1);
    return VGICP_OK;
}

vgicp_status vgicp_memory_in_use(vgicp_ctx *ctx, int64_t *bytes)
{
    if (!ctx || !bytes) return VGICP_ERR_INVALID_ARG;
    *bytes = ctx->bytes_in_use;
    return VGICP_OK;
}

vgicp_status vgicp_kernel_launches(vgicp_ctx *ctx, int64_t *count)
{
    if (!ctx || !count) return VGICP_ERR_INVALID_ARG;
    *count = ctx->launches;
    return VGICP_OK;
}

vgicp_status vgicp_kernel_timing(vgicp_ctx *ctx, int32_t kernel, double *total_ms, int64_t *launches)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (kernel < 0 || kernel > 2 || !total_ms) return fail(ctx, VGICP_ERR_INVALID_ARG, "kernel_timing: bad arguments");
    const Lane::KTimer &K = LN.ktimer[kernel];
    double sum = 0.0;
    for (int i = 0; i < K.used; ++i) {
        CU(cudaEventSynchronize(K.end[i]));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, K.begin[i], K.end[i]));
        sum += ms;
    }
    *total_ms = sum;
    if (launches) *launches = K.used;
    return VGICP_OK;
}

vgicp_status vgicp_kernel_timing_reset(vgicp_ctx *ctx)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    CU(cudaStreamSynchronize(LN.stream));   // no recorded event is still pending when its slot is reused
    for (Lane::KTimer &K : LN.ktimer) K.used = 0;
    return VGICP_OK;
}

const char *vgicp_last_error(const vgicp_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

const char *vgicp_status_string(vgicp_status s)
{
    switch (s) {
    case VGICP_OK: return "VGICP_OK";
    case VGICP_ERR_INVALID_ARG: return "VGICP_ERR_INVALID_ARG";
    case VGICP_ERR_OOM: return "VGICP_ERR_OOM";
    case VGICP_ERR_NOT_FOUND: return "VGICP_ERR_NOT_FOUND";
    case VGICP_ERR_EMPTY: return "VGICP_ERR_EMPTY";
    case VGICP_ERR_CUDA: return "VGICP_ERR_CUDA";
    case VGICP_ERR_TIMEOUT: return "VGICP_ERR_TIMEOUT";
    case VGICP_ERR_BUDGET: return "VGICP_ERR_BUDGET";
    case VGICP_ERR_NUMERIC: return "VGICP_ERR_NUMERIC";
    }
    return "unknown";
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Read-only access to a context for entry points in other translation units.
// ---------------------------------------------------------------------------
namespace vg {

bool ctx_view(vgicp_ctx *ctx, CtxView *v)
{
    if (!ctx || !v) return false;
    v->stream = LN.stream;
    v->device = ctx->device;
    v->num_sms = ctx->num_sms;
    v->chunk = default_chunk(ctx->opt);
    v->variant = ctx->opt.linearize_variant;
    v->linearize_cull = ctx->opt.linearize_cull;
    v->compensated = ctx->opt.precision == VGICP_PREC_F32_COMP;
    v->neighbors = neighbor_count(ctx->opt);
    v->count_weighted = ctx->opt.count_weighted;
    v->linearize_cull = lin_cull(ctx->opt);
    v->blocks_per_sm = ctx->opt.blocks_per_sm;
    v->d_maps = ctx->d_maps;
    v->d_frames = ctx->d_frames;
    return true;
}

bool ctx_is_map(vgicp_ctx *ctx, int64_t handle) { return lookup(ctx, handle, Obj::MAP) != nullptr; }

bool ctx_frame_size(vgicp_ctx *ctx, int64_t handle, int64_t *n)
{
    Obj *o = lookup(ctx, handle, Obj::FRAME);
    if (!o) return false;
    *n = o->n;
    return true;
}

vgicp_status ctx_fail(vgicp_ctx *ctx, vgicp_status s, const char *msg) { return fail(ctx, s, "%s", msg); }

void ctx_count_launches(vgicp_ctx *ctx, int n) { ctx->launches += n; }

int ctx_add_frames_gather(vgicp_ctx *ctx, const float *const *points, const float *const *covs,
                                   const int64_t *n, int64_t m, int64_t *out)
{
    if (m <= 0) return VGICP_OK;
    int64_t total = 0;
    for (int64_t u = 0; u < m; ++u) {
        if (n[u] < 0 || n[u] > ((int64_t)1 << 31) - 1 || (n[u] > 0 && (!points[u] || !covs[u])))
            return fail(ctx, VGICP_ERR_INVALID_ARG, "add_frames: frame %lld: bad size or pointer", (long long)u);
        total += n[u];
    }
    // each frame's arrays copied to its place in the lane's staging buffer
    const size_t pb = align256((size_t)total * 12);
    TRY(ensure(ctx, LN.ws_stage, pb + (size_t)total * 24));
    char *base = (char *)LN.ws_stage.p;
    int64_t o = 0;
    for (int64_t u = 0; u < m; ++u) {
        TRY(h2d(ctx, base + 12 * o, points[u], (size_t)n[u] * 12));
        TRY(h2d(ctx, base + pb + 24 * o, covs[u], (size_t)n[u] * 24));
        o += n[u];
    }
    return add_frames_staged(ctx, (const float *)base, (const float *)(base + pb), n, m, total, out);
}

bool ctx_descs(vgicp_ctx *ctx, int64_t map, int64_t frame, MapDesc *m, FrameDesc *f, int64_t *n_points)
{
    uint32_t mi, fi;
    if (!lookup(ctx, map, Obj::MAP, &mi)) return false;
    Obj *fo = lookup(ctx, frame, Obj::FRAME, &fi);
    if (!fo) return false;
    *m = ctx->h_maps[mi];
    *f = ctx->h_frames[fi];
    *n_points = fo->n;
    return true;
}

}  // namespace vg
