// Voxel overlap (Eq. 7-8): the number of source points whose transformed point
// falls in an existing target voxel.  Only the floor decision matters here, so
// each axis uses a plain float32 fma chain on the split translation with a
// proven per-pair error bound; the points that bound cannot decide take the
// float32-pair transform, and the float64 reference only if that too is
// undecided (points on voxel faces).
#include <algorithm>

#include "kernels.cuh"

namespace vg {

namespace {

__device__ __noinline__ bool point_key_slow(const PoseParam &P, const MapDesc &m, float px, float py, float pz,
                                           int k[3])
{
    bool decided = true;
    float d[3], rp[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        decided &= axis_key_ff(P.Rh + 3 * a, P.Rl + 3 * a, P.th[a], P.tl[a], px, py, pz, m.r_h, m.r_l, m.inv_rf,
                               P.ffm[a], P.ffup[a], k[a], d[a], rp[a]);
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

// Overlap matrix.  A work item is (slice of kSlice sources, one target): the
// CTA stages the target's compact presence table (32-bit keys relative to its
// voxel box, capacity ~2x its voxel count) in shared memory once, then streams
// the slice's live sources through it, kPPT points per thread per step.  Only
// items with a pair that survives culling are listed (k_overlap_items) in
// tiers of decreasing size, each tier in slice-major order up to warp
// interleaving.  CTAs take them from that list through a global counter, so
// the CTAs in flight share one slice of sources (a few MB, L2-resident) while
// each holds a different target table, no SM sits idle while another works
// through a long static share, and the items that start last are short.  Targets without a
// compact table that fits (very large or very wide maps) probe the main table
// in global memory instead; undecided floors take the slower exact path.
constexpr int kOvBlock = 1024, kPPT = 4, kSlice = 16;
constexpr int kSmemLog2 = 15;   // 32,768 compact keys = 128 KB of shared memory

// Shared-memory words of the small CTAs (two 512-thread CTAs per SM, 64 KB
// each) and of the large ones (one 1024-thread CTA per SM, 128 KB).
constexpr int kSmallWords = 16384;


// Items are fetched in tiers of decreasing size (live cull chunks of the
// item: at least kTierChunks[0], then kTierChunks[1], ..., then the rest), so
// the last items to start are short ones and the CTAs finish close together.
constexpr int kTiers = 4;
__device__ __constant__ int kTierChunks[kTiers - 1] = {192, 96, 48};
constexpr int kHdrInts = 16;   // per list: kTiers counts and the fetch counter

// List the (slice, target) items with at least one pair not culled, in two
// lists by the target's presence structure: one that fits kSmallWords words
// (list A) or not (list B).  Tier t of list k occupies entries
// list + (k kTiers + t) total ...; list k's header hdr[(kTiers + 1) k ..] holds
// the tiers' counts and the fetch counter (zeroed first).
__global__ void k_overlap_items(const PoseParam *__restrict__ pairs, const MapDesc *__restrict__ maps, int n_src,
                                int n_tgt, int32_t *__restrict__ list, int *__restrict__ hdr)
{
    const int n_slices = (n_src + kSlice - 1) / kSlice;
    const int64_t total = (int64_t)n_slices * n_tgt;
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool live = false, small = false;
    int chunks = 0;
    if (v < total) {
        const int sl = (int)(v / n_tgt), t = (int)(v - (int64_t)sl * n_tgt);
        const int s0 = sl * kSlice, s1 = min(n_src, s0 + kSlice);
        for (int s = s0; s < s1; ++s) {
            const PoseParam &P = pairs[(int64_t)s * n_tgt + t];
            if (!__ldg(&P.cull)) {
                live = true;
                chunks += __popc(__ldg(&P.cmask));
            }
        }
        if (live) {
            const int32_t *cm = maps[__ldg(&pairs[(int64_t)s0 * n_tgt + t].map)].cmeta;
            small = (cm[2] && cm[3] <= kSmallWords) || (cm[1] && (1 << cm[0]) <= kSmallWords);
        }
    }
    const unsigned lane = threadIdx.x & 31;
    int tier = kTiers - 1;
#pragma unroll
    for (int t = kTiers - 2; t >= 0; --t)
        if (chunks >= kTierChunks[t]) tier = t;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
#pragma unroll
        for (int t = 0; t < kTiers; ++t) {
            const bool mine = live && (small == (k == 0)) && tier == t;
            const unsigned b = __ballot_sync(0xffffffffu, mine);
            int base = 0;
            if (lane == 0 && b) base = atomicAdd(hdr + (kTiers + 1) * k + t, __popc(b));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (mine) list[(int64_t)(k * kTiers + t) * total + base + __popc(b & ((1u << lane) - 1u))] = (int32_t)v;
        }
    }
}

template <int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_overlap_matrix(const PoseParam *__restrict__ pairs,
                                                                const MapDesc *__restrict__ maps,
                                                                const FrameDesc *__restrict__ frames, int n_src,
                                                                int n_tgt, const int32_t *__restrict__ list,
                                                                int *__restrict__ hdr, int smem_words,
                                                                unsigned long long *__restrict__ counts)
{
    extern __shared__ uint4 s_tab4[];
    const uint32_t *s_tab = (const uint32_t *)s_tab4;
    constexpr int PW = (int)(sizeof(PoseParam) / 4);
    __shared__ PoseParam sP[kSlice];
    __shared__ MapDesc sM;
    __shared__ int s_kb[6], s_lg, s_smem, s_words;   // voxel box, compact table size, staged: 1 table, 2 bitmap
    __shared__ const float4 *s_pa[kSlice];
    __shared__ const float *s_gb[kSlice];
    __shared__ int s_n[kSlice], s_csh[kSlice], s_next[kSlice];   // s_next: next round of each source
    __shared__ int s_q;
    const int lane = threadIdx.x & 31;
    int n_live = 0;
#pragma unroll
    for (int t = 0; t < kTiers; ++t) n_live += hdr[t];
    const int64_t total = (int64_t)((n_src + kSlice - 1) / kSlice) * n_tgt;
    for (;;) {
        __syncthreads();                                // previous item's readers are done
        if (threadIdx.x == 0) s_q = atomicAdd(hdr + kTiers, 1);
        __syncthreads();
        int q = s_q;
        if (q >= n_live) break;
        int tier = 0;
        while (tier < kTiers - 1 && q >= hdr[tier]) q -= hdr[tier++];   // uniform across the block
        const int64_t v = list[tier * total + q];
        const int sl = (int)(v / n_tgt), t = (int)(v - (int64_t)sl * n_tgt);
        const int s0 = sl * kSlice, ns = min(n_src, s0 + kSlice) - s0;
        // the slice's pair parameters (one warp per source) and the target's table
        for (int wib = threadIdx.x >> 5; wib < ns; wib += BLOCK / 32) {
            {
                const uint32_t *src = (const uint32_t *)(pairs + (int64_t)(s0 + wib) * n_tgt + t);
                uint32_t *dst = (uint32_t *)(sP + wib);
                for (int j = lane; j < PW; j += 32) dst[j] = __ldg(src + j);
                const PoseParam &Pg = pairs[(int64_t)(s0 + wib) * n_tgt + t];
                const FrameDesc &F = frames[__ldg((const int *)&Pg.frame)];
                if (lane == 0) {
                    s_next[wib] = 0;
                    s_pa[wib] = F.pa;
                    s_gb[wib] = F.gbox;
                    s_n[wib] = (int)F.n;
                    s_csh[wib] = F.cshift;
                }
            }
        }
        if (threadIdx.x == 0) {
            sM = maps[pairs[(int64_t)s0 * n_tgt + t].map];
            s_lg = sM.cmeta[0];
            s_words = sM.cmeta[3];
            s_smem = (sM.cmeta[2] && s_words <= smem_words) ? 2
                                                              : ((sM.cmeta[1] && (1 << s_lg) <= smem_words) ? 1 : 0);
#pragma unroll
            for (int j = 0; j < 6; ++j) s_kb[j] = sM.kbox[j];
        }
        __syncthreads();
        if (s_smem) {
            const uint4 *src = (const uint4 *)sM.ckeys;
            const int n4 = s_smem == 2 ? (s_words + 3) / 4 : (1 << s_lg) / 4;
            for (int i = threadIdx.x; i < n4; i += BLOCK) s_tab4[i] = __ldg(src + i);
        }
        __syncthreads();
        const MapDesc &m = sM;
        const int smem = s_smem;
        const uint32_t lg = (uint32_t)s_lg;
        const int ex = s_kb[3] - s_kb[0], ey = s_kb[4] - s_kb[1], ez = s_kb[5] - s_kb[2];
        for (int si = 0; si < ns; ++si) {
            const PoseParam &P = sP[si];
            if (P.cull) continue;                       // uniform across the block
            const float4 *__restrict__ pa = s_pa[si];
            const int n = s_n[si], csh = s_csh[si], ng = (n + kGroup - 1) / kGroup;
            unsigned int hits = 0;
            // rounds of 32 consecutive candidate groups, taken by the warps from a
            // per-source counter (no block barrier, no fixed shares): a candidate is
            // kept when in a live cull chunk and (with a group test) when reaching an
            // occupied coarse cell of the target; then the live ones, kPPT groups
            // per step, one lane per point
            for (;;) {
                int rnd = 0;
                if (lane == 0) rnd = atomicAdd(&s_next[si], 1);
                const int gr = __shfl_sync(0xffffffffu, rnd, 0) * 32;
                if (gr >= ng) break;
                const int gc = gr + lane;
                bool l = gc < ng && ((P.cmask >> (((int64_t)gc * kGroup) >> csh)) & 1u);
                if (l && P.cs >= 0) l = group_live(P, s_gb[si] + 6 * (int64_t)gc, m.r_h, m.inv_rf, m.coarse);
                uint32_t livem = __ballot_sync(0xffffffffu, l);
            while (livem) {
                float px[kPPT], py[kPPT], pz[kPPT];
                bool have[kPPT];
#pragma unroll
                for (int j = 0; j < kPPT; ++j) {
                    int i = n;
                    if (livem) {
                        i = (gr + __ffs(livem) - 1) * kGroup + lane;
                        livem &= livem - 1u;
                    }
                    have[j] = i < n;
                    const float4 A = have[j] ? __ldg(pa + i) : make_float4(0.f, 0.f, 0.f, 0.f);
                    px[j] = A.x; py[j] = A.y; pz[j] = A.z;
                }
                if (smem == 2) {
                    // presence bitmap: box test, then one bit; floors undecided at a face take the exact path
                    const uint32_t X = (uint32_t)ex + 1u, XY = X * ((uint32_t)ey + 1u);
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        int d[3];
                        bool dec = true;
#pragma unroll
                        for (int a = 0; a < 3; ++a)
                            dec &= axis_box(P.Rh + 3 * a, P.tfh[a], P.hm[a], P.koff[a], px[j], py[j], pz[j],
                                            m.inv_rf, d[a]);
                        const bool in = (unsigned)d[0] <= (unsigned)ex && (unsigned)d[1] <= (unsigned)ey &&
                                        (unsigned)d[2] <= (unsigned)ez;
                        const uint32_t bit = (uint32_t)d[0] + X * (uint32_t)d[1] + XY * (uint32_t)d[2];
                        const uint32_t word = (have[j] && dec && in) ? s_tab[bit >> 5] : 0xFFFFFFFFu;
                        hits += ((word >> (bit & 31)) & 1u) ^ 1u;
                        if (have[j] && !dec) {
                            int k[3];
                            hits += point_key_slow(P, m, px[j], py[j], pz[j], k) &&
                                    probe(m.keys, m.mask, m.log2cap, pack_key(k[0], k[1], k[2])) >= 0;
                        }
                    }
                } else if (smem) {
                    // keys of all points first, then all first probes, then the rare chains
                    uint32_t ck[kPPT], slot[kPPT];
                    int state[kPPT];                    // 0 no, 1 yes, 2 probing, 3 undecided floor
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        int d[3];
                        bool dec = true;
#pragma unroll
                        for (int a = 0; a < 3; ++a)
                            dec &= axis_box(P.Rh + 3 * a, P.tfh[a], P.hm[a], P.koff[a], px[j], py[j], pz[j],
                                            m.inv_rf, d[a]);
                        const bool in = (unsigned)d[0] <= (unsigned)ex && (unsigned)d[1] <= (unsigned)ey &&
                                        (unsigned)d[2] <= (unsigned)ez;
                        state[j] = !have[j] ? 0 : (!dec ? 3 : (in ? 2 : 0));
                        ck[j] = pack_compact(d[0], d[1], d[2]);
                        slot[j] = hash_compact(ck[j], lg);
                    }
                    uint32_t first[kPPT];
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) first[j] = (state[j] == 2) ? s_tab[slot[j]] : kEmptyCompact;
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        if (state[j] == 2) {
                            if (first[j] == ck[j]) state[j] = 1;
                            else if (first[j] == kEmptyCompact) state[j] = 0;
                            else {
                                const uint32_t mask = (1u << lg) - 1u;
                                uint32_t s = (slot[j] + 1) & mask;
                                state[j] = 0;
                                for (uint32_t q = 0; q < mask; ++q) {
                                    const uint32_t v = s_tab[s];
                                    if (v == ck[j]) { state[j] = 1; break; }
                                    if (v == kEmptyCompact) break;
                                    s = (s + 1) & mask;
                                }
                            }
                        } else if (state[j] == 3) {     // face: float32-pair, then float64
                            int k[3];
                            state[j] = point_key_slow(P, m, px[j], py[j], pz[j], k) &&
                                               probe(m.keys, m.mask, m.log2cap, pack_key(k[0], k[1], k[2])) >= 0
                                           ? 1
                                           : 0;
                        }
                        hits += (state[j] == 1);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) {
                        int k[3];
                        bool dec = true, hit = false;
#pragma unroll
                        for (int a = 0; a < 3; ++a)
                            dec &= axis_key_split(P.Rh + 3 * a, P.tfh[a], P.tol[a], P.rup[a], P.k0[a], px[j],
                                                  py[j], pz[j], m.r_h, m.r_l, m.inv_rf, k[a]);
                        if (have[j] && dec && k[0] != INT32_MIN && k[1] != INT32_MIN && k[2] != INT32_MIN)
                            hit = probe(m.keys, m.mask, m.log2cap, pack_key(k[0], k[1], k[2])) >= 0;
                        if (have[j] && !dec)
                            hit = point_key_slow(P, m, px[j], py[j], pz[j], k) &&
                                  probe(m.keys, m.mask, m.log2cap, pack_key(k[0], k[1], k[2])) >= 0;
                        hits += hit;
                    }
                }
            }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) hits += __shfl_xor_sync(0xffffffffu, hits, o);
            if (lane == 0 && hits)
                atomicAdd(counts + (int64_t)(s0 + si) * n_tgt + t, (unsigned long long)hits);
        }
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
        float d[3], rp[3];
        bool decided = true;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            decided &= axis_key_ff(P.Rh + 3 * a, P.Rl + 3 * a, P.th[a], P.tl[a], A.x, A.y, A.z, m.r_h, m.r_l,
                                   m.inv_rf, P.ffm[a], P.ffup[a], k[a], d[a], rp[a]);
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

// out[0] += pairs not culled, out[1] += the points the matrix kernel visits for
// them (points of the live groups of live chunks); one warp per pair.
__global__ void k_count_live(const PoseParam *__restrict__ pairs, int64_t n_pairs,
                             const FrameDesc *__restrict__ frames, const MapDesc *__restrict__ maps,
                             unsigned long long *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long live = 0, pts = 0;
    for (int64_t g = w0; g < n_pairs; g += nw) {
        const PoseParam &P = pairs[g];
        if (P.cull) continue;
        live += lane == 0;
        const FrameDesc &F = frames[P.frame];
        const MapDesc &m = maps[P.map];
        const int64_t ng = (F.n + kGroup - 1) / kGroup;
        for (int64_t q = lane; q < ng; q += 32) {
            bool l = (P.cmask >> ((q * kGroup) >> F.cshift)) & 1u;
            if (l && P.cs >= 0) l = group_live(P, F.gbox + 6 * q, m.r_h, m.inv_rf, m.coarse);
            if (l) pts += (unsigned long long)min((int64_t)kGroup, F.n - q * kGroup);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        live += __shfl_xor_sync(0xffffffffu, live, o);
        pts += __shfl_xor_sync(0xffffffffu, pts, o);
    }
    if (lane == 0 && (live || pts)) {
        atomicAdd(out, live);
        atomicAdd(out + 1, pts);
    }
}

}  // namespace

void launch_count_live(const PoseParam *pairs, int64_t n_pairs, const FrameDesc *frames, const MapDesc *maps,
                       unsigned long long *out, cudaStream_t st)
{
    if (n_pairs <= 0) return;
    k_count_live<<<148 * 8, 256, 0, st>>>(pairs, n_pairs, frames, maps, out);
}

void launch_overlap(const PoseParam *params, const MapDesc *maps, const FrameDesc *frames, const WorkItem *items,
                    int n_items, unsigned long long *counts, int grid, cudaStream_t st)
{
    if (n_items <= 0) return;
    k_overlap<<<grid, 256, 0, st>>>(params, maps, frames, items, n_items, counts);
}

size_t overlap_matrix_scratch_bytes(int n_src, int n_tgt)
{
    const int64_t n_slices = (n_src + kSlice - 1) / kSlice;
    return (size_t)(2 * kTiers * n_slices * n_tgt + kHdrInts) * sizeof(int32_t);
}

void launch_overlap_matrix(const PoseParam *pairs, const MapDesc *maps, const FrameDesc *frames, int n_src,
                           int n_tgt, unsigned long long *counts, void *scratch, int num_sms,
                           cudaStream_t st)
{
    if (n_src <= 0 || n_tgt <= 0) return;
    int *hdr = (int *)scratch;
    int32_t *list = (int32_t *)scratch + kHdrInts;
    const int64_t total = (int64_t)((n_src + kSlice - 1) / kSlice) * n_tgt;
    cudaMemsetAsync(hdr, 0, kHdrInts * sizeof(int), st);
    k_overlap_items<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(pairs, maps, n_src, n_tgt, list, hdr);
    // items whose target's table fits 64 KB: two 512-thread CTAs per SM, each
    // with its own item and staged table; the others one 1024-thread CTA per SM
    // with up to 128 KB (an empty list's kernel exits at once)
    {
        const int smem = kSmallWords * 4;
        cudaFuncSetAttribute(k_overlap_matrix<512, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_overlap_matrix<512, 2><<<num_sms * 2, 512, smem, st>>>(pairs, maps, frames, n_src, n_tgt, list, hdr,
                                                                  kSmallWords, counts);
    }
    {
        const int words = 1 << kSmemLog2, smem = words * 4;
        cudaFuncSetAttribute(k_overlap_matrix<kOvBlock, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_overlap_matrix<kOvBlock, 1><<<num_sms, kOvBlock, smem, st>>>(pairs, maps, frames, n_src, n_tgt,
                                                                     list + kTiers * total, hdr + kTiers + 1, words,
                                                                     counts);
    }
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
