// Frame packing and the batched voxelmap build (Sec. III-A: a voxel's
// distribution aggregates the distributions of the points that fall in it:
// mean of the point means and mean of the point covariances).
//
// Build of all maps of a batch in four launches:
//   clear      keys <- EMPTY, voxel counters <- 0, presence words reset
//   insert     per point: voxel key, atomicCAS into the map's open-addressing
//              table; the thread that claims a slot takes a dense voxel id and
//              zeroes that voxel's accumulators
//   accumulate per point: exact fixed-point sums (int64 atomics, so the result
//              does not depend on the order the GPU runs the points in)
//   finalize   per voxel: mean relative to the voxel's lower corner, mean
//              covariance, count -> the slot's 48 B record; its 32-bit key
//              relative to the map's voxel box into a presence table sized by
//              the voxel count (overlap queries stage it in shared memory) and
//              its bit in the coarse occupancy bitmap
#include <algorithm>
#include "kernels.cuh"

namespace vg {

namespace {

constexpr int kAcc = 10;   // count, 3 mean sums, 6 covariance sums

// Re-lay the points and covariances and gather the frame statistics (stats
// must hold the initial values: zeros, then +inf minima and -inf maxima).
__global__ void k_frame_pack(const float *__restrict__ pts, const float *__restrict__ cov, int64_t n,
                             float4 *__restrict__ pa, float4 *__restrict__ pb, float *__restrict__ pc,
                             unsigned int *stats)
{
    float m = 0.f, am[3] = {0.f, 0.f, 0.f};
    uint32_t mn[3] = {kOrderedPosInf, kOrderedPosInf, kOrderedPosInf};
    uint32_t mx[3] = {kOrderedNegInf, kOrderedNegInf, kOrderedNegInf};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float *p = pts + 3 * i, *c = cov + 6 * i;
        pa[i] = make_float4(p[0], p[1], p[2], c[0]);
        pb[i] = make_float4(c[1], c[2], c[3], c[4]);
        pc[i] = c[5];
#pragma unroll
        for (int j = 0; j < 6; ++j) m = fmaxf(m, fabsf(c[j]));
        if (isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2])) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                am[j] = fmaxf(am[j], fabsf(p[j]));
                mn[j] = min(mn[j], ordered_bits(p[j]));
                mx[j] = max(mx[j], ordered_bits(p[j]));
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            am[j] = fmaxf(am[j], __shfl_xor_sync(0xffffffffu, am[j], o));
            mn[j] = min(mn[j], __shfl_xor_sync(0xffffffffu, mn[j], o));
            mx[j] = max(mx[j], __shfl_xor_sync(0xffffffffu, mx[j], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        if (m > 0.f) atomicMax(stats + kStatCmax, __float_as_uint(m));
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (am[j] > 0.f) atomicMax(stats + kStatPmax + j, __float_as_uint(am[j]));
            atomicMin(stats + kStatMin + j, mn[j]);
            atomicMax(stats + kStatMax + j, mx[j]);
        }
    }
}

// Batched frame registration: frame u's n points start at src_off[u] of the
// staged point / covariance arrays; its descriptor is in the table at index
// fidx[u].  Items are (frame, start, count) chunks of points.
__global__ void k_frames_init(const int32_t *__restrict__ fidx, int m, const FrameDesc *__restrict__ frames)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= m) return;
    unsigned int *st = (unsigned int *)frames[fidx[u]].stats;
    st[kStatCmax] = 0u;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        st[kStatPmax + j] = 0u;
        st[kStatMin + j] = kOrderedPosInf;
        st[kStatMax + j] = kOrderedNegInf;
    }
}

// mode 0: write the streams in the given order and gather the statistics;
// mode 1: statistics only; mode 2: write the streams in the frame's stored
// point order (stream position i takes given point perm[i]; a frame without a
// perm array, one of at most one point, in the given order), no statistics.
__global__ void k_frames_pack(const float *__restrict__ pts, const float *__restrict__ cov,
                              const int64_t *__restrict__ src_off, const int32_t *__restrict__ fidx,
                              const WorkItem *__restrict__ items, int n_items, const FrameDesc *__restrict__ frames,
                              int mode)
{
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const WorkItem w = items[it];
        const FrameDesc F = frames[fidx[w.unit]];
        const float *p0 = pts + 3 * src_off[w.unit], *c0 = cov + 6 * src_off[w.unit];
        if (mode == 2) {
            for (int k = threadIdx.x; k < w.count; k += blockDim.x) {
                const int64_t i = w.start + k, j = F.perm ? (int64_t)F.perm[i] : i;   // one-point frames: no perm
                const float *p = p0 + 3 * j, *c = c0 + 6 * j;
                ((float4 *)F.pa)[i] = make_float4(p[0], p[1], p[2], c[0]);
                ((float4 *)F.pb)[i] = make_float4(c[1], c[2], c[3], c[4]);
                ((float *)F.pc)[i] = c[5];
            }
            continue;
        }
        float m = 0.f, am[3] = {0.f, 0.f, 0.f};
        uint32_t mn[3] = {kOrderedPosInf, kOrderedPosInf, kOrderedPosInf};
        uint32_t mx[3] = {kOrderedNegInf, kOrderedNegInf, kOrderedNegInf};
        for (int k = threadIdx.x; k < w.count; k += blockDim.x) {
            const int64_t i = w.start + k;
            const float *p = p0 + 3 * i, *c = c0 + 6 * i;
            if (mode == 0) {
                ((float4 *)F.pa)[i] = make_float4(p[0], p[1], p[2], c[0]);
                ((float4 *)F.pb)[i] = make_float4(c[1], c[2], c[3], c[4]);
                ((float *)F.pc)[i] = c[5];
            }
#pragma unroll
            for (int j = 0; j < 6; ++j) m = fmaxf(m, fabsf(c[j]));
            if (isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2])) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    am[j] = fmaxf(am[j], fabsf(p[j]));
                    mn[j] = min(mn[j], ordered_bits(p[j]));
                    mx[j] = max(mx[j], ordered_bits(p[j]));
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                am[j] = fmaxf(am[j], __shfl_xor_sync(0xffffffffu, am[j], o));
                mn[j] = min(mn[j], __shfl_xor_sync(0xffffffffu, mn[j], o));
                mx[j] = max(mx[j], __shfl_xor_sync(0xffffffffu, mx[j], o));
            }
        }
        if ((threadIdx.x & 31) == 0) {
            unsigned int *st = (unsigned int *)F.stats;
            if (m > 0.f) atomicMax(st + kStatCmax, __float_as_uint(m));
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (am[j] > 0.f) atomicMax(st + kStatPmax + j, __float_as_uint(am[j]));
                atomicMin(st + kStatMin + j, mn[j]);
                atomicMax(st + kStatMax + j, mx[j]);
            }
        }
    }
}

// Spatial point order of frames (one block per frame at a time): each finite
// point's cell in a grid of 256^3 cubic cells spanning the frame's bounding
// box (cell edge = the largest box extent / 256), the cells in Morton order
// (z-order: bits of x, y, z interleaved), points of one cell in their given
// order, points that are not finite last.  A stable LSD radix sort of the
// 24-bit codes, 8 bits per pass: per pass a digit histogram and its prefix,
// then tiles of kSortBlock points in index order, each point's rank among the
// tile's points of its digit from the warps' __match_any_sync groups and the
// per-warp counts.  The result is a permutation (perm[i] = given index of the
// point stored at i): deterministic, so a cloud registered twice is stored
// the same way.  Scratch: 4 arrays of total-points uint32 (keys and indices,
// two buffers), frame u's points at src_off[u].
constexpr int kSortBlock = 256, kSortBins = 256, kSortWarps = kSortBlock / 32;

__device__ __forceinline__ uint32_t spread3(uint32_t v)
{
    // bit b of v to bit 3 b (v < 256)
    v &= 0xffu;
    v = (v | (v << 8)) & 0x0000f00fu;
    v = (v | (v << 4)) & 0x000c30c3u;
    v = (v | (v << 2)) & 0x00249249u;
    return v;
}

__global__ void __launch_bounds__(kSortBlock) k_frames_order(const float *__restrict__ pts,
                                                             const int64_t *__restrict__ src_off,
                                                             const int32_t *__restrict__ fidx, int m,
                                                             const FrameDesc *__restrict__ frames,
                                                             uint32_t *__restrict__ scratch, int64_t total)
{
    __shared__ uint32_t s_cnt[kSortWarps][kSortBins];
    __shared__ uint32_t s_base[kSortBins], s_tot[kSortBins];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (int u = blockIdx.x; u < m; u += gridDim.x) {
        const FrameDesc F = frames[fidx[u]];
        const int64_t n = F.n, off = src_off[u];
        if (!F.perm || n == 0) continue;
        uint32_t *keyA = scratch + off, *idxA = scratch + total + off;
        uint32_t *keyB = scratch + 2 * total + off, *idxB = scratch + 3 * total + off;
        float lo[3], ext = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = from_ordered_bits(((const uint32_t *)F.stats)[kStatMin + a]);
            const float hi = from_ordered_bits(((const uint32_t *)F.stats)[kStatMax + a]);
            ext = fmaxf(ext, hi - lo[a]);
        }
        const float inv = ext > 0.f ? 256.f / ext : 0.f;
        const float *p0 = pts + 3 * off;
        for (int64_t i = t; i < n; i += kSortBlock) {
            const float *p = p0 + 3 * i;
            uint32_t code = 0xffffffu;
            if (isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2])) {
                uint32_t q[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float c = fmaxf(0.f, (p[a] - lo[a]) * inv);
                    q[a] = c < 255.f ? (uint32_t)c : 255u;
                }
                code = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
            }
            keyA[i] = code;
            idxA[i] = (uint32_t)i;
        }
        __syncthreads();
        for (int pass = 0; pass < 3; ++pass) {
            const int sh = 8 * pass;
            const uint32_t *sk = pass == 1 ? keyB : keyA, *si = pass == 1 ? idxB : idxA;
            uint32_t *dk = pass == 1 ? keyA : keyB, *di = pass == 1 ? idxA : idxB;
            // digit histogram and its exclusive prefix
            if (t < kSortBins) s_tot[t] = 0u;
            for (int j = t; j < kSortWarps * kSortBins; j += kSortBlock) (&s_cnt[0][0])[j] = 0u;
            __syncthreads();
            for (int64_t i = t; i < n; i += kSortBlock) atomicAdd(&s_tot[(sk[i] >> sh) & 0xffu], 1u);
            __syncthreads();
            if (t < 32) {
                uint32_t run = 0;
                for (int q = 0; q < kSortBins / 32; ++q) {
                    const uint32_t v = s_tot[q * 32 + t];
                    uint32_t x = v;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                        if (lane >= o) x += y;
                    }
                    s_base[q * 32 + t] = run + x - v;
                    run += __shfl_sync(0xffffffffu, x, 31);
                }
            }
            __syncthreads();
            for (int64_t b = 0; b < n; b += kSortBlock) {
                const int64_t i = b + t;
                const bool ok = i < n;
                const uint32_t key = ok ? sk[i] : 0u, id = ok ? si[i] : 0u;
                const uint32_t d = ok ? ((key >> sh) & 0xffu) : 0x100u;   // 0x100: past the end
                const uint32_t peers = __match_any_sync(0xffffffffu, d);
                const uint32_t rank = __popc(peers & lt);
                if (ok && rank == 0) s_cnt[w][d] = (uint32_t)__popc(peers);
                __syncthreads();
                if (t < kSortBins) {            // per digit: exclusive prefix over the warps
                    uint32_t run = 0;
                    for (int q = 0; q < kSortWarps; ++q) {
                        const uint32_t c = s_cnt[q][t];
                        s_cnt[q][t] = run;
                        run += c;
                    }
                    s_tot[t] = run;
                }
                __syncthreads();
                if (ok) {
                    const uint32_t pos = s_base[d] + s_cnt[w][d] + rank;
                    dk[pos] = key;
                    di[pos] = id;
                }
                __syncthreads();
                if (t < kSortBins) s_base[t] += s_tot[t];
                for (int j = t; j < kSortWarps * kSortBins; j += kSortBlock) (&s_cnt[0][0])[j] = 0u;
                __syncthreads();
            }
        }
        // three passes: A -> B -> A -> B
        for (int64_t i = t; i < n; i += kSortBlock) ((int32_t *)F.perm)[i] = (int32_t)idxB[i];
        __syncthreads();
    }
}

// Spatial point order within tiles: every registration item (4,096 consecutive
// given points of one frame, one block) sorted on its own by the same 24-bit
// Morton cell codes as k_frames_order (cells over the whole frame's box),
// ties by given index: a bitonic sort of 4,096 unique 64-bit keys (code,
// index) in shared memory.  Points stay within their tile, so a frame of any
// size is ordered by as many blocks as it has tiles.
constexpr int kTileSort = 4096, kTileBlock = 1024;

__global__ void __launch_bounds__(kTileBlock) k_frames_order_tiles(const float *__restrict__ pts,
                                                                   const int64_t *__restrict__ src_off,
                                                                   const int32_t *__restrict__ fidx,
                                                                   const WorkItem *__restrict__ items, int n_items,
                                                                   const FrameDesc *__restrict__ frames)
{
    __shared__ unsigned long long s_key[kTileSort];
    const int t = threadIdx.x;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const WorkItem w = items[it];
        const FrameDesc F = frames[fidx[w.unit]];
        if (!F.perm) continue;                          // uniform: the whole block
        float lo[3], ext = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = from_ordered_bits(((const uint32_t *)F.stats)[kStatMin + a]);
            const float hi = from_ordered_bits(((const uint32_t *)F.stats)[kStatMax + a]);
            ext = fmaxf(ext, hi - lo[a]);
        }
        const float inv = ext > 0.f ? 256.f / ext : 0.f;
        const float *p0 = pts + 3 * (src_off[w.unit] + w.start);
        __syncthreads();                                // the previous item's readers are done
        for (int j = t; j < kTileSort; j += kTileBlock) {
            unsigned long long key = ~0ull;             // padding sorts last
            if (j < w.count) {
                const float *p = p0 + 3 * j;
                uint32_t code = 0xffffffu;
                if (isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2])) {
                    uint32_t q[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float c = fmaxf(0.f, (p[a] - lo[a]) * inv);
                        q[a] = c < 255.f ? (uint32_t)c : 255u;
                    }
                    code = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
                }
                key = ((unsigned long long)code << 32) | (unsigned long long)j;
            }
            s_key[j] = key;
        }
        __syncthreads();
        for (int k = 2; k <= kTileSort; k <<= 1)
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int i = t; i < kTileSort; i += kTileBlock) {
                    const int l = i ^ jj;
                    if (l > i) {
                        const unsigned long long a = s_key[i], b = s_key[l];
                        const bool up = (i & k) == 0;
                        if ((a > b) == up) {
                            s_key[i] = b;
                            s_key[l] = a;
                        }
                    }
                }
                __syncthreads();
            }
        for (int j = t; j < w.count; j += kTileBlock)
            ((int32_t *)F.perm)[w.start + j] = (int32_t)(w.start + (int64_t)(s_key[j] & 0xffffffffull));
    }
}

// Group boxes of many frames (after the streams are written): for every group of
// kGroup consecutive stored points the box of its finite points (min > max when
// it has none), one warp per group, over the point items (their starts are
// multiples of kGroup).
__global__ void k_frames_group_boxes(const int32_t *__restrict__ fidx, const WorkItem *__restrict__ items,
                                     int n_items, const FrameDesc *__restrict__ frames)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const WorkItem w = items[it];
        const FrameDesc F = frames[fidx[w.unit]];
        for (int g = wib; g * kGroup < w.count; g += nw) {
            const int64_t i = w.start + (int64_t)g * kGroup + lane;
            float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
            if (i < w.start + w.count) {
                const float4 p = F.pa[i];
                if (isfinite(p.x) && isfinite(p.y) && isfinite(p.z)) {
                    mn[0] = mx[0] = p.x;
                    mn[1] = mx[1] = p.y;
                    mn[2] = mx[2] = p.z;
                }
            }
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    mn[j] = fminf(mn[j], __shfl_xor_sync(0xffffffffu, mn[j], o));
                    mx[j] = fmaxf(mx[j], __shfl_xor_sync(0xffffffffu, mx[j], o));
                }
            if (lane < 6) {
                const int64_t grp = (w.start >> 5) + g;
                ((float *)F.gbox)[6 * grp + lane] = lane < 3 ? mn[lane] : mx[lane - 3];
            }
        }
    }
}

// Chunk boxes of many frames: item (frame, chunk) per block, as k_chunk_boxes.
__global__ void k_frames_chunk_boxes(const int32_t *__restrict__ fidx, const WorkItem *__restrict__ chunks,
                                     int n_chunks, const FrameDesc *__restrict__ frames)
{
    __shared__ float s[6][8];
    for (int it = blockIdx.x; it < n_chunks; it += gridDim.x) {
        const WorkItem w = chunks[it];      // start = chunk index
        const FrameDesc F = frames[fidx[w.unit]];
        const int c = (int)w.start;
        const int64_t b = (int64_t)c << F.cshift, e = min(F.n, b + ((int64_t)1 << F.cshift));
        float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
            const float4 p = F.pa[i];
            if (isfinite(p.x) && isfinite(p.y) && isfinite(p.z)) {
                mn[0] = fminf(mn[0], p.x); mn[1] = fminf(mn[1], p.y); mn[2] = fminf(mn[2], p.z);
                mx[0] = fmaxf(mx[0], p.x); mx[1] = fmaxf(mx[1], p.y); mx[2] = fmaxf(mx[2], p.z);
            }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn[j] = fminf(mn[j], __shfl_xor_sync(0xffffffffu, mn[j], o));
                mx[j] = fmaxf(mx[j], __shfl_xor_sync(0xffffffffu, mx[j], o));
            }
        const int wq = threadIdx.x >> 5;
        __syncthreads();                                // previous item's readers are done
        if ((threadIdx.x & 31) == 0) {
#pragma unroll
            for (int j = 0; j < 3; ++j) { s[j][wq] = mn[j]; s[3 + j][wq] = mx[j]; }
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            float v = s[threadIdx.x][0];
            for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
                v = threadIdx.x < 3 ? fminf(v, s[threadIdx.x][q]) : fmaxf(v, s[threadIdx.x][q]);
            ((float *)F.cbox)[6 * c + threadIdx.x] = v;
        }
    }
}

__global__ void k_scatter_frame_descs(const uint32_t *__restrict__ idx, const FrameDesc *__restrict__ src, int n,
                                      FrameDesc *__restrict__ table)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) table[idx[i]] = src[i];
}

// Bounding box of each cull chunk of a frame (finite points only; an empty
// chunk gets min > max).  One block per chunk.
__global__ void k_chunk_boxes(const float4 *__restrict__ pa, int64_t n, int shift, float *__restrict__ cbox)
{
    const int c = blockIdx.x;
    const int64_t b = (int64_t)c << shift, e = min(n, b + ((int64_t)1 << shift));
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
        const float4 p = pa[i];
        if (isfinite(p.x) && isfinite(p.y) && isfinite(p.z)) {
            mn[0] = fminf(mn[0], p.x); mn[1] = fminf(mn[1], p.y); mn[2] = fminf(mn[2], p.z);
            mx[0] = fmaxf(mx[0], p.x); mx[1] = fmaxf(mx[1], p.y); mx[2] = fmaxf(mx[2], p.z);
        }
    }
    __shared__ float s[6][8];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn[j] = fminf(mn[j], __shfl_xor_sync(0xffffffffu, mn[j], o));
            mx[j] = fmaxf(mx[j], __shfl_xor_sync(0xffffffffu, mx[j], o));
        }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int j = 0; j < 3; ++j) { s[j][w] = mn[j]; s[3 + j][w] = mx[j]; }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        float v = s[threadIdx.x][0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
            v = threadIdx.x < 3 ? fminf(v, s[threadIdx.x][q]) : fmaxf(v, s[threadIdx.x][q]);
        cbox[6 * c + threadIdx.x] = v;
    }
}

// Empty tables, one block per map: keys and compact presence entries in
// 16-byte stores (capacities are powers of two >= 16, so every array holds a
// whole number of vectors), the coarse occupancy words, the voxel count and
// the box.  The slot -> voxel id array needs no clearing: only slots claimed
// in this build are ever read from it.
__global__ void k_build_clear(const MapDesc *__restrict__ maps, const BuildUnit *__restrict__ units, int n_units)
{
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const BuildUnit U = units[u];
        const MapDesc &m = maps[U.map];
        const int64_t cap = (int64_t)m.mask + 1;
        uint4 *keys = (uint4 *)m.keys, *ck = (uint4 *)m.ckeys;
        const uint4 ones = make_uint4(~0u, ~0u, ~0u, ~0u);
        for (int64_t v = threadIdx.x; v < cap / 2; v += blockDim.x) keys[v] = ones;   // kEmptyKey = all ones
        for (int64_t v = threadIdx.x; v < cap / 4; v += blockDim.x) ck[v] = ones;     // kEmptyCompact = all ones
        for (int v = threadIdx.x; v < kCoarseWords; v += blockDim.x) m.coarse[v] = 0u;
        if (threadIdx.x == 0) {
            *U.n_voxels = 0;
            m.kbox[0] = m.kbox[1] = m.kbox[2] = INT32_MAX;
            m.kbox[3] = m.kbox[4] = m.kbox[5] = INT32_MIN;
        }
    }
}

// Voxel coordinate of a point of the map's own frame (identity pose).
// Power-of-two resolutions: p * inv_r and floor are exact in float32.
// Otherwise: the float64 reference floor(p * inv_r).
__device__ __forceinline__ bool own_key(const MapDesc &m, float px, float py, float pz, int k[3])
{
    if (m.pow2) {
        const float f[3] = {floorf(px * m.inv_rf), floorf(py * m.inv_rf), floorf(pz * m.inv_rf)};
        bool ok = true;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            ok = ok && (f[i] >= (float)kKeyMin && f[i] <= (float)kKeyMax);
            k[i] = ok ? (int)f[i] : 0;
        }
        return ok;
    }
    const double T[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    double q[3];
    return key_f64(T, px, py, pz, m.inv_r, k, q);
}

__global__ void k_build_insert(const MapDesc *__restrict__ maps, const FrameDesc *__restrict__ frames,
                               const BuildUnit *__restrict__ units, const WorkItem *__restrict__ items, int n_items,
                               BuildScratch scr)
{
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const WorkItem w = items[it];
        const BuildUnit u = units[w.unit];
        const MapDesc m = maps[u.map];
        const FrameDesc f = frames[u.frame];
        for (int64_t i = w.start + threadIdx.x; i < w.start + w.count; i += blockDim.x) {
            const float4 a = __ldg(f.pa + i);
            int k[3];
            int32_t slot = -1;
            if (own_key(m, a.x, a.y, a.z, k)) {
                const uint64_t key = pack_key(k[0], k[1], k[2]);
                uint32_t s = hash_slot(key, m.log2cap);
                for (uint32_t t = 0; t <= m.mask; ++t) {
                    // a plain read first: a slot's key never changes once set, so a
                    // key read here is final and only an empty slot needs the CAS
                    // (points of one voxel mostly find their key already there)
                    const uint64_t seen = __ldcg(m.keys + s);
                    if (seen == key) {
                        slot = (int32_t)s;
                        break;
                    }
                    if (seen != kEmptyKey) {
                        s = (s + 1) & m.mask;
                        continue;
                    }
                    const unsigned long long old =
                        atomicCAS((unsigned long long *)(m.keys + s), (unsigned long long)kEmptyKey,
                                  (unsigned long long)key);
                    if (old == kEmptyKey) {          // claimed: this thread owns the new voxel
                        const int32_t vid = (int32_t)atomicAdd(u.n_voxels, 1u);
                        scr.vid_of_slot[u.slot_base + s] = vid;
                        scr.slot_of_vid[u.point_base + vid] = (int32_t)s;
                        int64_t *acc = scr.acc + (u.point_base + vid) * kAcc;
#pragma unroll
                        for (int j = 0; j < kAcc; ++j) acc[j] = 0;
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            atomicMin(m.kbox + j, k[j]);
                            atomicMax(m.kbox + 3 + j, k[j]);
                        }
                        slot = (int32_t)s;
                        break;
                    }
                    if (old == key) { slot = (int32_t)s; break; }
                    s = (s + 1) & m.mask;
                }
            }
            scr.slot_of_point[u.point_base + i] = slot;
        }
    }
}

__device__ __forceinline__ float cov_scale(const float *stats)
{
    const float c = stats[kStatCmax];
    if (!(c > 0.f)) return 1.f;
    int e;
    frexpf(c, &e);                 // c < 2^e
    return ldexpf(1.f, 40 - e);    // |entry| * scale < 2^40
}

__device__ __forceinline__ float mean_scale(const MapDesc &m) { return m.inv_rf * 0x1p32f; }

__global__ void __launch_bounds__(256) k_build_accumulate(const MapDesc *__restrict__ maps,
                                                          const FrameDesc *__restrict__ frames,
                                                          const BuildUnit *__restrict__ units,
                                                          const WorkItem *__restrict__ items, int n_items,
                                                          BuildScratch scr)
{
    __shared__ long long s_stage[8][kAcc - 1][32];    // per warp of the 256-thread block
    long long(*stage)[32] = s_stage[threadIdx.x >> 5];
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const WorkItem w = items[it];
        const BuildUnit u = units[w.unit];
        const MapDesc m = maps[u.map];
        const FrameDesc f = frames[u.frame];
        const float sc = cov_scale(f.stats), sm = mean_scale(m);
        const unsigned lane = threadIdx.x & 31;
        // whole warps step together (lanes of one voxel are grouped below)
        for (int64_t i0 = w.start + (threadIdx.x & ~31u); i0 < w.start + w.count; i0 += blockDim.x) {
            const int64_t i = i0 + lane;
            int32_t vid = -1;
            long long v[kAcc];
#pragma unroll
            for (int j = 0; j < kAcc; ++j) v[j] = 0;
            if (i < w.start + w.count) {
                const int32_t slot = scr.slot_of_point[u.point_base + i];
                if (slot >= 0) {
                    vid = scr.vid_of_slot[u.slot_base + slot];
                    const float4 a = __ldg(f.pa + i), b = __ldg(f.pb + i);
                    const float c22 = __ldg(f.pc + i);
                    // the point's own voxel coordinate (the key it was inserted under):
                    // recomputed where that is three float32 floors (power-of-two r),
                    // else read from the slot
                    int kx, ky, kz;
                    if (m.pow2) {
                        int k[3];
                        own_key(m, a.x, a.y, a.z, k);
                        kx = k[0];
                        ky = k[1];
                        kz = k[2];
                    } else {
                        unpack_key(m.keys[slot], kx, ky, kz);
                    }
                    // offset from the voxel's lower corner k r, r = r_h + r_l
                    const float dx = __fmaf_rn(-(float)kx, m.r_l, __fmaf_rn(-(float)kx, m.r_h, a.x));
                    const float dy = __fmaf_rn(-(float)ky, m.r_l, __fmaf_rn(-(float)ky, m.r_h, a.y));
                    const float dz = __fmaf_rn(-(float)kz, m.r_l, __fmaf_rn(-(float)kz, m.r_h, a.z));
                    v[0] = 1;
                    v[1] = __float2ll_rn(dx * sm);
                    v[2] = __float2ll_rn(dy * sm);
                    v[3] = __float2ll_rn(dz * sm);
                    v[4] = __float2ll_rn(a.w * sc);
                    v[5] = __float2ll_rn(b.x * sc);
                    v[6] = __float2ll_rn(b.y * sc);
                    v[7] = __float2ll_rn(b.z * sc);
                    v[8] = __float2ll_rn(b.w * sc);
                    v[9] = __float2ll_rn(c22 * sc);
                }
            }
            // the lanes of one voxel (a spatially ordered frame keeps them close):
            // the lowest adds up their sums from shared memory and makes the one
            // set of int64 atomics.  Integer sums: the result does not depend on
            // the grouping or on the order the atomics land in.
            const unsigned peers = __match_any_sync(0xffffffffu, vid);
            const int leader = __ffs(peers) - 1;
#pragma unroll
            for (int j = 1; j < kAcc; ++j) stage[j - 1][lane] = v[j];
            __syncwarp();
            if ((int)lane == leader && vid >= 0) {
                for (unsigned rest = peers & (peers - 1u); rest; rest &= rest - 1u) {
                    const int b = __ffs(rest) - 1;
#pragma unroll
                    for (int j = 1; j < kAcc; ++j) v[j] += stage[j - 1][b];
                }
                v[0] = __popc(peers);
                unsigned long long *acc = (unsigned long long *)(scr.acc + (u.point_base + vid) * kAcc);
#pragma unroll
                for (int j = 0; j < kAcc; ++j) atomicAdd(acc + j, (unsigned long long)v[j]);
            }
            __syncwarp();
        }
    }
}

__global__ void k_build_finalize(const MapDesc *__restrict__ maps, const FrameDesc *__restrict__ frames,
                                 const BuildUnit *__restrict__ units, const WorkItem *__restrict__ items,
                                 int n_items, BuildScratch scr)
{
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const WorkItem w = items[it];
        const BuildUnit u = units[w.unit];
        const MapDesc m = maps[u.map];
        const FrameDesc f = frames[u.frame];
        const uint32_t nv = *u.n_voxels;
        const int *kb = m.kbox;
        const bool ok = nv > 0 && kb[3] - kb[0] <= kCompactMaxX && kb[4] - kb[1] <= kCompactMaxX &&
                        kb[5] - kb[2] <= kCompactMaxZ;
        uint32_t lg = 4;
        while (lg < m.log2cap && (1u << lg) < 4u * nv) ++lg;
        const uint64_t X = nv > 0 ? (uint64_t)(kb[3] - kb[0] + 1) : 0, Y = nv > 0 ? (uint64_t)(kb[4] - kb[1] + 1) : 0,
                       Z = nv > 0 ? (uint64_t)(kb[5] - kb[2] + 1) : 0;
        const uint64_t words = (X * Y * Z + 31) / 32;
        const bool bitmap = ok && words <= (uint64_t)(m.mask + 1) && words <= kBitmapMaxWords;
        // coarse occupancy: the smallest shift >= 2 whose grid fits kCoarseWords words
        int cs = 2;
        uint64_t cx = 0, cy = 0, cz = 0;
        if (nv > 0) {
            for (;; ++cs) {
                cx = (uint64_t)((kb[3] - kb[0]) >> cs) + 1;
                cy = (uint64_t)((kb[4] - kb[1]) >> cs) + 1;
                cz = (uint64_t)((kb[5] - kb[2]) >> cs) + 1;
                if (cx * cy * cz <= (uint64_t)kCoarseWords * 32) break;
            }
        }
        if (w.start == 0 && threadIdx.x == 0) {
            m.cmeta[0] = (int32_t)lg;
            m.cmeta[1] = (ok && !bitmap) ? 1 : 0;
            m.cmeta[2] = bitmap ? 1 : 0;
            m.cmeta[3] = bitmap ? (int32_t)words : 0;
            m.cmeta[4] = nv > 0 ? cs : -1;
            m.cmeta[5] = (int32_t)cx;
            m.cmeta[6] = (int32_t)cy;
            m.cmeta[7] = (int32_t)cz;
        }
        const float isc = 1.f / cov_scale(f.stats), ism = 1.f / mean_scale(m);
        const uint32_t cmask = (1u << lg) - 1u;
        // the item's share of the map's voxels: the same fraction of [0, nv) as
        // its points are of the frame (the items tile the points, so the shares
        // tile the voxels; nv <= f.n), so every item of the map finalizes about
        // the same number of voxels
        const int64_t v0 = f.n > 0 ? w.start * (int64_t)nv / f.n : 0;
        const int64_t v1 = f.n > 0 ? (w.start + w.count) * (int64_t)nv / f.n : 0;
        for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
            const int64_t *acc = scr.acc + (u.point_base + v) * kAcc;
            const int32_t slot = scr.slot_of_vid[u.point_base + v];
            const float n = (float)acc[0], in = 1.f / n;
            VoxelRec r;
            r.a = make_float4(__ll2float_rn(acc[1]) * ism * in, __ll2float_rn(acc[2]) * ism * in,
                              __ll2float_rn(acc[3]) * ism * in, __ll2float_rn(acc[4]) * isc * in);
            r.b = make_float4(__ll2float_rn(acc[5]) * isc * in, __ll2float_rn(acc[6]) * isc * in,
                              __ll2float_rn(acc[7]) * isc * in, __ll2float_rn(acc[8]) * isc * in);
            r.c = make_float4(__ll2float_rn(acc[9]) * isc * in, __uint_as_float((uint32_t)acc[0]), 0.f, 0.f);
            m.rec[slot] = r;
            int kx, ky, kz;
            unpack_key(m.keys[slot], kx, ky, kz);
            const uint64_t cbit = (uint64_t)((kx - kb[0]) >> cs) +
                                  cx * ((uint64_t)((ky - kb[1]) >> cs) + cy * (uint64_t)((kz - kb[2]) >> cs));
            atomicOr(m.coarse + (cbit >> 5), 1u << (cbit & 31));
            if (!ok) continue;
            if (bitmap) {
                const uint64_t bit =
                    (uint64_t)(kx - kb[0]) + X * ((uint64_t)(ky - kb[1]) + Y * (uint64_t)(kz - kb[2]));
                atomicAnd(m.ckeys + (bit >> 5), ~(1u << (bit & 31)));
                continue;
            }
            const uint32_t ck = pack_compact(kx - kb[0], ky - kb[1], kz - kb[2]);
            uint32_t s = hash_compact(ck, lg);
            for (uint32_t t = 0; t <= cmask; ++t) {
                const uint32_t old = atomicCAS(m.ckeys + s, kEmptyCompact, ck);
                if (old == kEmptyCompact || old == ck) break;
                s = (s + 1) & cmask;
            }
        }
    }
}

// Shared-memory images of the listed maps (one block per map), made on first
// use by the shared-memory linearisation: the occupied slots are counted, and a
// map that qualifies gets its compact key table, voxel ids and dense records;
// every listed map's header is written (one that does not qualify is marked
// invalid).  Voxel ids follow the order the slots are claimed in; lookups see
// the same records whatever that order.
constexpr int kImgBuildBlock = 512;

__global__ void __launch_bounds__(kImgBuildBlock) k_map_image(const MapDesc *__restrict__ maps,
                                                              const int32_t *__restrict__ idx, int n)
{
    __shared__ uint32_t s_cnt, s_next;
    for (int u = blockIdx.x; u < n; u += gridDim.x) {
        const MapDesc m = maps[idx[u]];
        const uint32_t cap = m.mask + 1u;
        if (threadIdx.x == 0) {
            s_cnt = 0u;
            s_next = 0u;
        }
        __syncthreads();
        uint32_t c = 0;
        for (uint32_t s = threadIdx.x; s < cap; s += blockDim.x) c += __ldg(m.keys + s) != kEmptyKey;
        c = __reduce_add_sync(0xffffffffu, c);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_cnt, c);
        __syncthreads();
        const uint32_t nv = s_cnt;
        int kb[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) kb[j] = m.kbox[j];
        uint32_t *hdr = (uint32_t *)m.img;
        const bool ok = nv > 0 && nv <= (uint32_t)kImgMaxVoxels && kb[3] - kb[0] <= kCompactMaxX &&
                        kb[4] - kb[1] <= kCompactMaxX && kb[5] - kb[2] <= kCompactMaxZ;
        int lg = 4;
        while ((1u << lg) < 2u * nv) ++lg;
        if (threadIdx.x == 0) {
            hdr[0] = ok ? 1u : 0u;
            hdr[1] = (uint32_t)lg;
            hdr[2] = nv;
            hdr[3] = ok ? (uint32_t)(kb[3] - kb[0]) | ((uint32_t)(kb[4] - kb[1]) << 16) : 0u;   // box extents x, y
            for (int j = 0; j < 3; ++j) hdr[4 + j] = (uint32_t)kb[j];
            hdr[7] = ok ? (uint32_t)(kb[5] - kb[2]) : 0u;                                       // and z
        }
        if (ok) {
            uint32_t *keys = (uint32_t *)(m.img + kImgHeader);
            uint16_t *vids = (uint16_t *)(m.img + kImgHeader + ((size_t)4 << lg));
            float *recs = (float *)(m.img + kImgHeader + img_table_bytes(lg));
            const uint32_t mask = (1u << lg) - 1u;
            for (uint32_t t = threadIdx.x; t <= mask; t += blockDim.x) keys[t] = kEmptyCompact;
            __syncthreads();
            for (uint32_t s = threadIdx.x; s < cap; s += blockDim.x) {
                const uint64_t key = __ldg(m.keys + s);
                if (key == kEmptyKey) continue;
                const uint32_t v = atomicAdd(&s_next, 1u);
                int kx, ky, kz;
                unpack_key(key, kx, ky, kz);
                const uint32_t ck = pack_compact(kx - kb[0], ky - kb[1], kz - kb[2]);
                uint32_t h = hash_compact(ck, (uint32_t)lg);
                for (uint32_t t = 0; t <= mask; ++t) {
                    const uint32_t old = atomicCAS(keys + h, kEmptyCompact, ck);
                    if (old == kEmptyCompact) break;
                    h = (h + 1) & mask;
                }
                vids[h] = (uint16_t)v;
                const VoxelRec r = m.rec[s];
                float *o = recs + (size_t)v * kImgRecFloats;
                o[0] = r.a.x; o[1] = r.a.y; o[2] = r.a.z; o[3] = r.a.w;
                o[4] = r.b.x; o[5] = r.b.y; o[6] = r.b.z; o[7] = r.b.w;
                o[8] = r.c.x; o[9] = r.c.y;
            }
        }
        __syncthreads();                                // before the block's next map resets the counters
    }
}

__global__ void k_scatter_map_descs(const uint32_t *__restrict__ idx, const MapDesc *__restrict__ src, int n,
                                    MapDesc *__restrict__ table)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) table[idx[i]] = src[i];
}

__global__ void k_export(const MapDesc *__restrict__ mp, uint32_t cap, uint32_t *counter, uint64_t *keys_out,
                         VoxelRec *rec_out)
{
    const MapDesc m = *mp;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += gridDim.x * blockDim.x) {
        const uint64_t k = m.keys[s];
        if (k == kEmptyKey) continue;
        const uint32_t i = atomicAdd(counter, 1u);
        keys_out[i] = k;
        rec_out[i] = m.rec[s];
    }
}

}  // namespace

void launch_frame_pack(const float *points, const float *covs, int64_t n, float4 *pa, float4 *pb, float *pc,
                       float *stats, cudaStream_t st)
{
    if (n <= 0) return;
    const int block = 256;
    int grid = (int)((n + block - 1) / block);
    if (grid > 148 * 16) grid = 148 * 16;
    k_frame_pack<<<grid, block, 0, st>>>(points, covs, n, pa, pb, pc, (unsigned int *)stats);
}

void launch_frames_register(const float *pts, const float *cov, const int64_t *src_off, const int32_t *fidx, int m,
                            const WorkItem *items, int n_items, const WorkItem *chunks, int n_chunks,
                            const uint32_t *desc_idx, const FrameDesc *descs, FrameDesc *table, uint32_t *order_scratch,
                            int64_t total, int num_sms, int order_mode, cudaStream_t st)
{
    if (m <= 0) return;
    k_scatter_frame_descs<<<(m + 127) / 128, 128, 0, st>>>(desc_idx, descs, m, table);
    k_frames_init<<<(m + 127) / 128, 128, 0, st>>>(fidx, m, table);
    const int pg = std::min(n_items, 148 * 16);
    if (n_items > 0 && order_mode != 0) {
        // statistics (the bounding box), the spatial order, then the streams in that order
        k_frames_pack<<<pg, 256, 0, st>>>(pts, cov, src_off, fidx, items, n_items, table, 1);
        if (order_mode == 2)
            k_frames_order_tiles<<<std::min(n_items, num_sms * 2), kTileBlock, 0, st>>>(pts, src_off, fidx, items,
                                                                                     n_items, table);
        else
            k_frames_order<<<std::min(m, num_sms * 4), kSortBlock, 0, st>>>(pts, src_off, fidx, m, table,
                                                                            order_scratch, total);
        k_frames_pack<<<pg, 256, 0, st>>>(pts, cov, src_off, fidx, items, n_items, table, 2);
    } else if (n_items > 0) {
        k_frames_pack<<<pg, 256, 0, st>>>(pts, cov, src_off, fidx, items, n_items, table, 0);
    }
    if (n_items > 0) k_frames_group_boxes<<<pg, 256, 0, st>>>(fidx, items, n_items, table);
    if (n_chunks > 0)
        k_frames_chunk_boxes<<<std::min(n_chunks, 148 * 16), 256, 0, st>>>(fidx, chunks, n_chunks, table);
}

void launch_chunk_boxes(const float4 *pa, int64_t n, int shift, int nchunks, float *cbox, cudaStream_t st)
{
    if (nchunks <= 0) return;
    k_chunk_boxes<<<nchunks, 256, 0, st>>>(pa, n, shift, cbox);
}

void launch_voxelmap_build(const MapDesc *maps, const FrameDesc *frames, const BuildUnit *units, int n_units,
                           const WorkItem *items, int n_items, BuildScratch scr, int grid, cudaStream_t st)
{
    if (n_units <= 0) return;
    k_build_clear<<<std::min(n_units, 148 * 8), 512, 0, st>>>(maps, units, n_units);
    if (n_items > 0) {
        k_build_insert<<<grid, 256, 0, st>>>(maps, frames, units, items, n_items, scr);
        k_build_accumulate<<<grid, 256, 0, st>>>(maps, frames, units, items, n_items, scr);
        k_build_finalize<<<grid, 256, 0, st>>>(maps, frames, units, items, n_items, scr);
    }
}

void launch_map_images(const MapDesc *maps, const int32_t *idx, int n, int num_sms, cudaStream_t st)
{
    if (n <= 0) return;
    k_map_image<<<std::min(n, num_sms * 4), kImgBuildBlock, 0, st>>>(maps, idx, n);
}

void launch_scatter_map_descs(const uint32_t *idx, const MapDesc *src, int n, MapDesc *table, cudaStream_t st)
{
    if (n <= 0) return;
    k_scatter_map_descs<<<(n + 127) / 128, 128, 0, st>>>(idx, src, n, table);
}

void launch_export_voxels(const MapDesc *map_dev, uint32_t cap, uint32_t *counter, uint64_t *keys_out,
                          VoxelRec *rec_out, cudaStream_t st)
{
    int grid = (int)((cap + 255) / 256);
    if (grid > 148 * 8) grid = 148 * 8;
    k_export<<<grid, 256, 0, st>>>(map_dev, cap, counter, keys_out, rec_out);
}

}  // namespace vg
