// Voxel overlap (Eq. 7-8): the number of source points whose transformed point
// falls in an existing target voxel.  Only the floor decision matters here, so
// each axis uses a plain float32 fma chain on the split translation with a
// proven per-pair error bound; the points that bound cannot decide take the
// float32-pair transform, and the float64 reference only if that too is
// undecided (points on voxel faces).
#include "kernels.cuh"

namespace vg {

namespace {

__device__ __noinline__ bool point_key_slow(const PoseParam &P, const MapDesc &m, float px, float py, float pz,
                                           int k[3])
{
    bool decided = true;
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        decided &= axis_key_ff(P.Rh + 3 * a, P.Rl + 3 * a, P.th[a], P.tl[a], px, py, pz, m.r_h, m.r_l, m.inv_rf,
                               P.ffm[a], P.ffup[a], k[a], d[a]);
    if (decided) return k[0] != INT32_MIN && k[1] != INT32_MIN && k[2] != INT32_MIN;
    double q[3];
    return key_f64(P.T, px, py, pz, m.inv_r, k, q);
}

__device__ __forceinline__ bool point_key_f32(const PoseParam &P, const MapDesc &m, float px, float py, float pz,
                                              int k[3])
{
    bool decided = true;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        decided &= axis_key_split(P.Rh + 3 * a, P.tfh[a], P.tol[a], P.rup[a], P.k0[a], px, py, pz, m.r_h, m.r_l,
                                  m.inv_rf, k[a]);
    if (decided) return k[0] != INT32_MIN && k[1] != INT32_MIN && k[2] != INT32_MIN;
    return point_key_slow(P, m, px, py, pz, k);
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
    if (sP.cull) return;          // uniform across the block
    const MapDesc m = sM;
    const float4 *__restrict__ pa = sPa + start;
    unsigned int hits = 0;
    for (int base = threadIdx.x & ~31; base < count; base += blockDim.x) {
        const int i = base + lane;
        bool hit = false;
        if (i < count) {
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

// Overlap matrix.  A work item is (chunk of 1,024 points of one source, tile
// of kTile targets): every thread keeps kPPT points in registers and, target by
// target, computes their voxel keys and issues their kPPT first hash probes back
// to back, so each thread has several independent loads in flight; collision
// chains (rare at load <= 2/3) and undecided floors take a slower path.
// Items are ordered target tile first, so the CTAs in flight share a few target
// tables while the source chunks stream through.
constexpr int kOvBlock = 256, kPPT = 4, kTile = 16, kOvChunk = kOvBlock * kPPT;

__global__ void __launch_bounds__(kOvBlock) k_overlap_matrix(const PoseParam *__restrict__ pairs,
                                                             const MapDesc *__restrict__ maps,
                                                             const FrameDesc *__restrict__ frames,
                                                             const WorkItem *__restrict__ chunks, int n_chunks,
                                                             int n_tgt, unsigned long long *__restrict__ counts)
{
    __shared__ PoseParam sP[kTile];
    __shared__ MapDesc sM[kTile];
    __shared__ unsigned int sHits[kTile];
    const int lane = threadIdx.x & 31;
    const int n_tiles = (n_tgt + kTile - 1) / kTile;
    const int64_t total = (int64_t)n_tiles * n_chunks;
    for (int64_t v = blockIdx.x; v < total; v += gridDim.x) {
        const int tt = (int)(v / n_chunks), c = (int)(v - (int64_t)tt * n_chunks);
        const WorkItem w = chunks[c];
        const int t0 = tt * kTile, nt = min(kTile, n_tgt - t0);
        __syncthreads();   // the previous item's readers of sP / sM / sHits are done
        int live = 0;
        if (threadIdx.x < nt) {
            sP[threadIdx.x] = pairs[(int64_t)w.unit * n_tgt + t0 + threadIdx.x];
            sM[threadIdx.x] = maps[sP[threadIdx.x].map];
            sHits[threadIdx.x] = 0;
            live = !sP[threadIdx.x].cull;
        }
        if (!__syncthreads_or(live)) continue;       // every pair of the tile culled: skip the points
        const float4 *__restrict__ pa = frames[sP[0].frame].pa + w.start;
        float px[kPPT], py[kPPT], pz[kPPT];
        bool have[kPPT];
#pragma unroll
        for (int j = 0; j < kPPT; ++j) {
            const int i = j * kOvBlock + threadIdx.x;
            have[j] = i < w.count;
            const float4 A = have[j] ? __ldg(pa + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            px[j] = A.x; py[j] = A.y; pz[j] = A.z;
        }
        for (int ti = 0; ti < nt; ++ti) {
            const PoseParam &P = sP[ti];
            if (P.cull) continue;                        // uniform across the block
            const MapDesc &m = sM[ti];
            const uint64_t *__restrict__ keys = m.keys;
            const uint32_t mask = m.mask, lg = m.log2cap;
            uint64_t key[kPPT];
            uint32_t slot[kPPT];
            int state[kPPT];                              // 0 miss, 1 hit, 2 probing, 3 undecided floor
#pragma unroll
            for (int j = 0; j < kPPT; ++j) {
                int k[3];
                bool dec = true;
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    dec &= axis_key_split(P.Rh + 3 * a, P.tfh[a], P.tol[a], P.rup[a], P.k0[a], px[j], py[j], pz[j],
                                          m.r_h, m.r_l, m.inv_rf, k[a]);
                const bool valid = k[0] != INT32_MIN && k[1] != INT32_MIN && k[2] != INT32_MIN;
                state[j] = !have[j] ? 0 : (!dec ? 3 : (valid ? 2 : 0));
                key[j] = valid ? pack_key(k[0], k[1], k[2]) : 0ull;
                slot[j] = hash_slot(key[j], lg);
            }
            uint64_t kv[kPPT];
#pragma unroll
            for (int j = 0; j < kPPT; ++j) kv[j] = (state[j] == 2) ? __ldg(keys + slot[j]) : kEmptyKey;
#pragma unroll
            for (int j = 0; j < kPPT; ++j) {
                if (state[j] != 2) continue;
                if (kv[j] == key[j]) state[j] = 1;
                else if (kv[j] == kEmptyKey) state[j] = 0;
                else {                                    // collision chain
                    state[j] = probe(keys, mask, lg, key[j]) >= 0 ? 1 : 0;
                }
            }
#pragma unroll
            for (int j = 0; j < kPPT; ++j) {
                if (state[j] == 3) {                      // face: float32-pair, then float64
                    int k[3];
                    state[j] = point_key_slow(P, m, px[j], py[j], pz[j], k) &&
                                       probe(keys, mask, lg, pack_key(k[0], k[1], k[2])) >= 0
                                   ? 1
                                   : 0;
                }
            }
            unsigned int h = 0;
#pragma unroll
            for (int j = 0; j < kPPT; ++j) h += __popc(__ballot_sync(0xffffffffu, state[j] == 1));
            if (lane == 0 && h) atomicAdd(sHits + ti, h);
        }
        __syncthreads();
        if (threadIdx.x < nt && sHits[threadIdx.x])
            atomicAdd(counts + (int64_t)w.unit * n_tgt + t0 + threadIdx.x, (unsigned long long)sHits[threadIdx.x]);
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
                                   m.inv_rf, P.ffm[a], P.ffup[a], k[a], d[a]);
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

int overlap_matrix_chunk() { return kOvChunk; }

void launch_overlap_matrix(const PoseParam *pairs, const MapDesc *maps, const FrameDesc *frames,
                           const WorkItem *chunks, int n_chunks, int n_tgt, unsigned long long *counts, int grid,
                           cudaStream_t st)
{
    if (n_chunks <= 0 || n_tgt <= 0) return;
    k_overlap_matrix<<<grid, kOvBlock, 0, st>>>(pairs, maps, frames, chunks, n_chunks, n_tgt, counts);
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
