// Voxel overlap (Eq. 7-8): the number of source points whose transformed point
// falls in an existing target voxel.  Only the floor decision matters here, so
// each axis uses a plain float32 fma chain with a proven error bound and only
// the points the bound cannot decide pay for the float64 reference.
#include "kernels.cuh"

namespace vg {

namespace {

__device__ __forceinline__ bool point_key_f32(const PoseParam &P, const MapDesc &m, float px, float py, float pz,
                                              int k[3])
{
    bool decided = true;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        decided &= axis_key_f32(P.Rh + 3 * a, P.th[a], px, py, pz, m.r_h, m.r_l, m.inv_rf, k[a]);
    if (decided) return k[0] != INT32_MIN && k[1] != INT32_MIN && k[2] != INT32_MIN;
    double q[3];
    return key_f64(P.T, px, py, pz, m.inv_r, k, q);
}

// Hits of points [start, start + count) of the pair's source in its target map,
// added to *count_out.  Called by whole blocks; whole warps iterate together so
// the ballot sees every lane.
__device__ __forceinline__ void overlap_item(const PoseParam *__restrict__ params, const MapDesc *__restrict__ maps,
                                             const FrameDesc *__restrict__ frames, int pair, int64_t start, int count,
                                             unsigned long long *count_out, PoseParam &sP, MapDesc &sM,
                                             const float4 *&sPa)
{
    const int lane = threadIdx.x & 31;
    __syncthreads();
    if (threadIdx.x == 0) {
        sP = params[pair];
        sM = maps[sP.map];
        sPa = frames[sP.frame].pa;
    }
    __syncthreads();
    const MapDesc m = sM;
    const float4 *__restrict__ pa = sPa;
    unsigned int hits = 0;
    const int64_t end = start + count;
    for (int64_t base = start + (threadIdx.x & ~31); base < end; base += blockDim.x) {
        const int64_t i = base + lane;
        bool hit = false;
        if (i < end) {
            const float4 A = __ldg(pa + i);
            int k[3];
            if (point_key_f32(sP, m, A.x, A.y, A.z, k))
                hit = probe(m.keys, m.mask, m.log2cap, pack_key(k[0], k[1], k[2])) >= 0;
        }
        hits += __popc(__ballot_sync(0xffffffffu, hit));
    }
    if (lane == 0 && hits) atomicAdd(count_out, (unsigned long long)hits);
}

__global__ void __launch_bounds__(256) k_overlap(const PoseParam *__restrict__ params,
                                                 const MapDesc *__restrict__ maps,
                                                 const FrameDesc *__restrict__ frames,
                                                 const WorkItem *__restrict__ items, int n_items,
                                                 unsigned long long *__restrict__ counts)
{
    __shared__ PoseParam sP;
    __shared__ MapDesc sM;
    __shared__ const float4 *sPa;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const WorkItem w = items[it];
        overlap_item(params, maps, frames, w.unit, w.start, w.count, counts + w.unit, sP, sM, sPa);
    }
}

__global__ void __launch_bounds__(256) k_overlap_matrix(const PoseParam *__restrict__ pairs,
                                                        const MapDesc *__restrict__ maps,
                                                        const FrameDesc *__restrict__ frames,
                                                        const WorkItem *__restrict__ chunks, int n_chunks, int n_tgt,
                                                        int tile, unsigned long long *__restrict__ counts)
{
    __shared__ PoseParam sP;
    __shared__ MapDesc sM;
    __shared__ const float4 *sPa;
    const int64_t per_tile = (int64_t)n_chunks * tile;
    const int64_t total = (int64_t)((n_tgt + tile - 1) / tile) * per_tile;
    for (int64_t v = blockIdx.x; v < total; v += gridDim.x) {
        const int64_t tt = v / per_tile, rem = v - tt * per_tile;
        const int c = (int)(rem / tile);
        const int t = (int)(tt * tile + rem % tile);
        if (t >= n_tgt) continue;   // uniform across the block
        const WorkItem w = chunks[c];
        const int pair = w.unit * n_tgt + t;
        overlap_item(pairs, maps, frames, pair, w.start, w.count, counts + pair, sP, sM, sPa);
    }
}

__global__ void k_correspondences(const PoseParam *__restrict__ prm, const MapDesc *__restrict__ maps,
                                  const FrameDesc *__restrict__ frames, int64_t n, int64_t *__restrict__ keys,
                                  int32_t *__restrict__ hit)
{
    const PoseParam &P = *prm;
    const MapDesc m = maps[P.map];
    const FrameDesc F = frames[P.frame];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 A = F.pa[i];
        // the batched linearisation's association: float32-pair transform, float64 at faces
        int k[3];
        float d[3];
        bool decided = true;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            decided &= axis_key_ff(P.Rh + 3 * a, P.Rl + 3 * a, P.th[a], P.tl[a], A.x, A.y, A.z, m.r_h, m.r_l,
                                   m.inv_rf, k[a], d[a]);
        bool ok;
        if (decided) {
            ok = k[0] != INT32_MIN && k[1] != INT32_MIN && k[2] != INT32_MIN;
        } else {
            double q[3];
            ok = key_f64(P.T, A.x, A.y, A.z, m.inv_r, k, q);
        }
        if (keys) {
#pragma unroll
            for (int a = 0; a < 3; ++a) keys[3 * i + a] = ok ? (int64_t)k[a] : INT64_MIN;
        }
        if (hit) hit[i] = ok ? (probe(m.keys, m.mask, m.log2cap, pack_key(k[0], k[1], k[2])) >= 0) : 0;
    }
}

}  // namespace

void launch_overlap(const PoseParam *params, const MapDesc *maps, const FrameDesc *frames, const WorkItem *items,
                    int n_items, unsigned long long *counts, int grid, cudaStream_t st)
{
    if (n_items <= 0) return;
    k_overlap<<<grid, 256, 0, st>>>(params, maps, frames, items, n_items, counts);
}

void launch_overlap_matrix(const PoseParam *pairs, const MapDesc *maps, const FrameDesc *frames,
                           const WorkItem *chunks, int n_chunks, int n_tgt, int tile, unsigned long long *counts,
                           int grid, cudaStream_t st)
{
    if (n_chunks <= 0 || n_tgt <= 0) return;
    k_overlap_matrix<<<grid, 256, 0, st>>>(pairs, maps, frames, chunks, n_chunks, n_tgt, tile, counts);
}

void launch_correspondences(const PoseParam *param, const MapDesc *maps, const FrameDesc *frames, int64_t n,
                            int64_t *keys, int32_t *hit, cudaStream_t st)
{
    if (n <= 0) return;
    int grid = (int)((n + 255) / 256);
    if (grid > 148 * 8) grid = 148 * 8;
    k_correspondences<<<grid, 256, 0, st>>>(param, maps, frames, n, keys, hit);
}

}  // namespace vg
