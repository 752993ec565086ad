// Linearisation of VGICP matching-cost factors (Eq. 3-6).
//
// Batched float32 path (one persistent launch for all factors)
//   With a = R p (the source point rotated into the target frame) and
//   J^t = [-[a]x, I], the paper's Jacobians factor as
//       J_B = J^t S,  S = [[I, 0], [-[t]x, I]],
//       J_A = -J^t D, D = blkdiag(R, R)
//   (q = a + t; R[p]x = [a]x R).  So every point only adds to
//       H^t = sum J^t' Omega J^t   (21 unique entries)
//       b^t = sum J^t' Omega e     (6)
//       cost = sum e' Omega e      (1)
//   and the per-factor 12x12 system is exactly
//       H = [[S' H^t S, -S' H^t D], [-D' H^t S, D' H^t D]],  b = [S' b^t ; -D' b^t],
//   formed once per factor in float64.  Accumulating about the translation
//   (lever arm a instead of q) keeps the float32 sums free of |t|-sized terms.
//   Per-point work is float32; the voxel floor and the residual offset inside
//   the voxel come from an error-free float32-pair transform (float64 fallback at
//   faces).  Each work item (a chunk of one factor's points) writes its 28 sums
//   as float64; a second kernel adds a factor's item sums in fixed order.
//
// Plain float64 path (one launch per factor)
//   Literal 3x12 Jacobian J = [-[q]x, I | R[p]x, -R], all 78 unique entries of
//   J' Omega J, 12 of J' Omega e and the cost, per point, in float64.
#include "kernels.cuh"
#include "vgicp.h"

namespace vg {

namespace {

constexpr int kNT = 28;   // accumulated values per point (batched path)

__device__ __forceinline__ void rel_pose(const double *__restrict__ TB, const double *__restrict__ TA, double *T)
{
    // T_BA = T_B^-1 T_A; every product and sum separately rounded, k = 0, 1, 2.
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) s = __dadd_rn(s, __dmul_rn(TB[4 * k + i], TA[4 * k + j]));
            T[4 * i + j] = s;
        }
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) s = __dadd_rn(s, __dmul_rn(TB[4 * k + i], __dsub_rn(TA[4 * k + 3], TB[4 * k + 3])));
        T[4 * i + 3] = s;
    }
}

__device__ __forceinline__ void split_pose(const double *T, PoseParam &p)
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double v = T[4 * i + j];
            const float h = __double2float_rn(v);
            p.Rh[3 * i + j] = h;
            p.Rl[3 * i + j] = __double2float_rn(v - (double)h);
        }
        const double v = T[4 * i + 3];
        const float h = __double2float_rn(v);
        p.th[i] = h;
        p.tl[i] = __double2float_rn(v - (double)h);
    }
}

// Live cull chunks of the source for this pair: chunk c's box (min/max of its
// points), moved by the pose, is tested against the target's voxel box.  The
// moved box is c' +- |R| h (centre, half extent) in float32, grown by 2^-18 of
// the magnitudes involved -- 16 times the float32 error of that evaluation --
// so a dead chunk provably holds no point that can find a voxel.
__device__ uint32_t chunk_mask(const PoseParam &p, const MapDesc &m, const FrameDesc &f)
{
    const int *kb = m.kbox;
    if (kb[0] > kb[3]) return 0u;
    const float blo[3] = {(float)((double)kb[0] * m.r), (float)((double)kb[1] * m.r), (float)((double)kb[2] * m.r)};
    const float bhi[3] = {(float)(((double)kb[3] + 1.0) * m.r), (float)(((double)kb[4] + 1.0) * m.r),
                          (float)(((double)kb[5] + 1.0) * m.r)};
    uint32_t mask = 0u;
    for (int c = 0; c < f.nchunks; ++c) {
        const float *b = f.cbox + 6 * c;
        if (!(b[0] <= b[3] && b[1] <= b[4] && b[2] <= b[5])) continue;    // no finite point
        const float cc[3] = {0.5f * (b[0] + b[3]), 0.5f * (b[1] + b[4]), 0.5f * (b[2] + b[5])};
        const float hh[3] = {0.5f * (b[3] - b[0]), 0.5f * (b[4] - b[1]), 0.5f * (b[5] - b[2])};
        bool live = true;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float ci = p.th[i], hi = 0.f, mag = fabsf(p.th[i]);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                ci = fmaf(p.Rh[3 * i + j], cc[j], ci);
                hi = fmaf(fabsf(p.Rh[3 * i + j]), hh[j], hi);
                mag = fmaf(fabsf(p.Rh[3 * i + j]), fabsf(cc[j]) + hh[j], mag);
            }
            const float mu = mag * 0x1p-18f + 1e-6f * (float)m.r + 1e-30f;
            live = live && (ci + hi + mu >= blo[i]) && (ci - hi - mu <= bhi[i]);
        }
        if (live) mask |= 1u << c;
    }
    return mask;
}

// The per-pair bounds of the float32 floors and, when asked, the exact culling
// tests, from p.T, the target map and the source frame's statistics.
__device__ void finish_param(PoseParam &p, const MapDesc &m, const FrameDesc &f, int cull)
{
    double pmax[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) pmax[j] = (double)f.stats[kStatPmax + j];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double t = p.T[4 * i + 3];
        const double Xr = fabs(p.T[4 * i]) * pmax[0] + fabs(p.T[4 * i + 1]) * pmax[1] + fabs(p.T[4 * i + 2]) * pmax[2];
        // split translation t = k0 r + tf (|tf| <= r / 2)
        double k0 = rint(t * m.inv_r);
        if (!(fabs(k0) < 4194304.0)) k0 = 0.0;   // |t| beyond 2^22 voxels: no split
        const double tf = t - k0 * m.r;
        p.k0[i] = (int32_t)k0;
        p.tfh[i] = __double2float_rn(tf);
        const double X = Xr + fabs(t), Xs = Xr + fabs(tf);
        const double tol = 0x1p-21 * Xs + 0x1p-22 * m.r + 0x1p-47 * X + 0x1p-100;
        p.tol[i] = __double2float_ru(tol);
        p.rup[i] = __double2float_rd((double)m.r_h - tol);
        // the same decision on y = x / r (overlap): tol in voxel units plus the
        // float32 rounding of y, of fl32(1/r) and of its fraction, with margin
        const double ty = tol * m.inv_r + 0x1p-21 * (Xs * m.inv_r + 1.0);
        p.hm[i] = ty < 0.5 ? __double2float_rd(0.5 - ty) : -1.f;
        const double fm = 0x1p-40 * X + 0x1p-100;
        p.ffm[i] = __double2float_ru(fm);
        p.ffup[i] = __double2float_rd((double)m.r_h - fm - 0x1p-22 * m.r);
    }
    p.cull = 0;
    p.cmask = f.nchunks >= 32 ? 0xffffffffu : ((1u << f.nchunks) - 1u);
    bool koff_ok = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const long long off = (long long)m.kbox[i] - (long long)p.k0[i];
        koff_ok = koff_ok && !(off > INT32_MAX / 2 || off < INT32_MIN / 2);
        p.koff[i] = (off > INT32_MAX / 2 || off < INT32_MIN / 2) ? INT32_MAX / 2 : (int32_t)off;
    }
    // group culling against the target's coarse occupancy (exact culling only)
    const int cs = m.cmeta[4];
    const bool coarse_ok = cull >= 2 && koff_ok && m.kbox[0] <= m.kbox[3] && cs >= 2 && cs < 31;
    p.cs = coarse_ok ? cs : -1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        p.bext[i] = coarse_ok ? m.kbox[3 + i] - m.kbox[i] : 0;
        p.cext[i] = coarse_ok ? m.cmeta[5 + i] : 0;
    }
    if (!cull) return;
    // A source without a finite point or a map without a voxel: nothing can hit.
    // Otherwise the float32 chunk boxes decide (every chunk dead: the pair is
    // culled); their bound is proven like the floors', and the pose test needs
    // no float64 (B300's float64 rate is a small fraction of float32's).
    const int *kb = m.kbox;
    bool finite = true;
#pragma unroll
    for (int j = 0; j < 3; ++j)
        finite = finite && from_ordered_bits(__float_as_uint(f.stats[kStatMin + j])) <=
                               from_ordered_bits(__float_as_uint(f.stats[kStatMax + j]));
    if (!finite || kb[0] > kb[3]) {
        p.cull = 1;
        p.cmask = 0u;
        return;
    }
    p.cmask = chunk_mask(p, m, f);
    if (p.cmask == 0u) p.cull = 1;
}

__global__ void k_prepare_factors(const int32_t *__restrict__ idx, int n_f, const double *__restrict__ poses,
                                  const MapDesc *__restrict__ maps, const FrameDesc *__restrict__ frames, int cull,
                                  PoseParam *__restrict__ out)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_f) return;
    PoseParam p;
    rel_pose(poses + 12 * (int64_t)idx[4 * f + 2], poses + 12 * (int64_t)idx[4 * f + 3], p.T);
    split_pose(p.T, p);
    p.map = idx[4 * f + 0];
    p.frame = idx[4 * f + 1];
    finish_param(p, maps[p.map], frames[p.frame], cull);
    out[f] = p;
}

// A float32 look at a pair before its float64 parameters: the relative pose in
// float32 (the translation difference taken in float64 first), the source's
// bounding box moved by it and grown by 2^-16 of the magnitudes involved (the
// float32 errors of the pose and of the moved box stay below 2^-20 of them),
// against the target's voxel box.  True when the grown box misses it on an
// axis, so no point of the pair can find a voxel; most pairs of an overlap
// matrix are such far pairs, and they skip the float64 work.
__device__ bool quick_cull(const double *__restrict__ TB, const double *__restrict__ TA, const MapDesc &m,
                           const FrameDesc &f)
{
    const int *kb = m.kbox;
    if (kb[0] > kb[3]) return true;                     // a map without voxels
    float mn[3], mx[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        mn[j] = from_ordered_bits(__float_as_uint(f.stats[kStatMin + j]));
        mx[j] = from_ordered_bits(__float_as_uint(f.stats[kStatMax + j]));
    }
    if (!(mn[0] <= mx[0] && mn[1] <= mx[1] && mn[2] <= mx[2])) return true;   // no finite point
    float d[3], dmax = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        d[k] = (float)(TA[4 * k + 3] - TB[4 * k + 3]);
        dmax = fmaxf(dmax, fabsf(d[k]));
    }
    const float rf = (float)m.r;
    bool miss = false;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float R[3], t = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float v = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) v = fmaf((float)TB[4 * k + i], (float)TA[4 * k + j], v);
            R[j] = v;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) t = fmaf((float)TB[4 * k + i], d[k], t);
        float c = t, h = 0.f, mag = fabsf(t);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float cc = 0.5f * (mn[j] + mx[j]), hh = 0.5f * (mx[j] - mn[j]);
            c = fmaf(R[j], cc, c);
            h = fmaf(fabsf(R[j]), hh, h);
            mag = fmaf(fabsf(R[j]), fabsf(cc) + hh, mag);
        }
        const float mu = (mag + dmax + 1.f) * 0x1p-16f + 1e-6f * rf + 1e-30f;
        const float blo = (float)((double)kb[i] * m.r), bhi = (float)(((double)kb[3 + i] + 1.0) * m.r);
        miss = miss || (c + h + mu < blo) || (c - h - mu > bhi);
    }
    return miss;
}

__global__ void k_prepare_pairs(const double *__restrict__ ps, const double *__restrict__ pt,
                                const int32_t *__restrict__ fidx, const int32_t *__restrict__ midx, int n_src,
                                int n_tgt, const MapDesc *__restrict__ maps, const FrameDesc *__restrict__ frames,
                                int cull, PoseParam *__restrict__ out)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)n_src * n_tgt) return;
    const int s = (int)(g / n_tgt), t = (int)(g % n_tgt);
    if (cull && quick_cull(pt + 12 * (int64_t)t, ps + 12 * (int64_t)s, maps[midx[t]], frames[fidx[s]])) {
        PoseParam q = {};
        q.map = midx[t];
        q.frame = fidx[s];
        q.cull = 1;
        q.cs = -1;
        out[g] = q;
        return;
    }
    PoseParam p;
    rel_pose(pt + 12 * (int64_t)t, ps + 12 * (int64_t)s, p.T);
    split_pose(p.T, p);
    p.map = midx[t];
    p.frame = fidx[s];
    finish_param(p, maps[p.map], frames[p.frame], cull);
    out[g] = p;
}

__global__ void k_prepare_list(const double *__restrict__ T, const int32_t *__restrict__ midx,
                               const int32_t *__restrict__ fidx, int n, const MapDesc *__restrict__ maps,
                               const FrameDesc *__restrict__ frames, int cull, PoseParam *__restrict__ out)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    PoseParam p;
#pragma unroll
    for (int i = 0; i < 12; ++i) p.T[i] = T[12 * (int64_t)g + i];
    split_pose(p.T, p);
    p.map = midx[g];
    p.frame = fidx[g];
    finish_param(p, maps[p.map], frames[p.frame], cull);
    out[g] = p;
}

__global__ void k_prepare_given(const double *__restrict__ T, int map, int frame, const MapDesc *__restrict__ maps,
                                const FrameDesc *__restrict__ frames, int cull, PoseParam *__restrict__ out)
{
    PoseParam p;
#pragma unroll
    for (int i = 0; i < 12; ++i) p.T[i] = T[i];
    split_pose(p.T, p);
    p.map = map;
    p.frame = frame;
    finish_param(p, maps[map], frames[frame], cull);
    *out = p;
}

// Voxel coordinate, in-voxel offset and lever arm R p of one point (batched path).
__device__ __forceinline__ bool point_key_ff(const PoseParam &P, const MapDesc &m, float px, float py, float pz,
                                             int k[3], float d[3], float rp[3])
{
    bool decided = true;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        decided &= axis_key_ff(P.Rh + 3 * a, P.Rl + 3 * a, P.th[a], P.tl[a], px, py, pz, m.r_h, m.r_l, m.inv_rf,
                               P.ffm[a], P.ffup[a], k[a], d[a], rp[a]);
    if (decided) return k[0] != INT32_MIN && k[1] != INT32_MIN && k[2] != INT32_MIN;
    double q[3];
    if (!key_f64(P.T, px, py, pz, m.inv_r, k, q)) return false;
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = __double2float_rn(q[a] - (double)k[a] * m.r);
    return true;
}

// Voxel coordinate, in-voxel offset and lever arm R p of one point from the
// plain float32 transform on the split translation t = k0 r + tf (the float32
// path's per-point transform).  The floor is exact: a point whose float32
// distance to a voxel face is within the proven error bound tol of the float64
// reference is left undecided and takes the float64 reference.  The offset and
// the lever arm carry float32 rounding (about 2^-22 of |R p| + |tf|).
__device__ __forceinline__ bool point_key_split(const PoseParam &P, const MapDesc &m, float px, float py, float pz,
                                                int k[3], float d[3], float rp[3])
{
    bool decided = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float *R = P.Rh + 3 * a;
        const float tf = P.tfh[a];
        const float x = __fmaf_rn(R[0], px, __fmaf_rn(R[1], py, __fmaf_rn(R[2], pz, tf)));
        const float kf = floorf(__fmul_rn(x, m.inv_rf));
        const float dd = __fmaf_rn(-kf, m.r_l, __fmaf_rn(-kf, m.r_h, x));
        decided &= (dd >= P.tol[a]) & (dd <= P.rup[a]);
        const int kk = (int)kf + P.k0[a];
        k[a] = (kk >= -kKeyOffset && kk <= kKeyOffset - 1) ? kk : INT32_MIN;
        d[a] = dd;
        rp[a] = __fsub_rn(x, tf);
    }
    if (decided) return k[0] != INT32_MIN && k[1] != INT32_MIN && k[2] != INT32_MIN;
    double q[3];
    if (!key_f64(P.T, px, py, pz, m.inv_r, k, q)) return false;
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = __double2float_rn(q[a] - (double)k[a] * m.r);
    return true;
}

// Slot of the voxel containing one source point, or -1; first probe issued by
// the caller so two points' probes can be in flight together.
struct PointSlot {
    uint64_t key;
    uint32_t h;
    bool ok;
};

template <bool FF>
__device__ __forceinline__ PointSlot point_hash(const PoseParam &P, const MapDesc &m, float px, float py, float pz,
                                                float d[3], float rp[3])
{
    int k[3];
    PointSlot r;
    r.ok = FF ? point_key_ff(P, m, px, py, pz, k, d, rp) : point_key_split(P, m, px, py, pz, k, d, rp);
    r.key = r.ok ? pack_key(k[0], k[1], k[2]) : 0ull;
    r.h = hash_slot(r.key, m.log2cap);
    return r;
}

template <class L = LdNC>
__device__ __forceinline__ int resolve_slot(const MapDesc &m, const PointSlot &ps, uint64_t first)
{
    if (!ps.ok || first == kEmptyKey) return -1;
    if (first == ps.key) return (int)ps.h;
    return probe_from<L>(m.keys, m.mask, ps.key, (ps.h + 1) & m.mask);
}

// Correspondence record of point j (CorrRecord layout); compiled in only for
// the recording instantiations.
template <bool REC>
__device__ __forceinline__ void record_point(const CorrRecord &rc, int64_t j, bool ok, uint64_t key, int32_t state)
{
    if constexpr (REC) {
        rc.key[j] = ok ? key : kEmptyKey;
        rc.state[j] = state;
    }
}

// The parts of a voxel record the linearisation reads (mean, covariance).
template <class L = LdNC>
__device__ __forceinline__ VoxelRec load_rec(const VoxelRec *r)
{
    VoxelRec v;
    v.a = L::ld(&r->a);
    v.b = L::ld(&r->b);
    v.c = make_float4(L::ld(&r->c.x), 0.f, 0.f, 0.f);
    return v;
}

// Residual e = mu_B - q (both relative to the voxel's lower corner), the
// information matrix Omega = (C_B + R C_A R^T)^-1 (Eq. 2, by the adjugate) and
// w = Omega e of one correspondence.  False when the combined covariance is not
// positive definite (the point then contributes nothing).
__device__ __forceinline__ bool point_omega(const float *R, const float4 &A, const float4 &B, float C22,
                                            const VoxelRec &v, const float d[3], float e[3], float o[6], float w[3])
{
    const float R0 = R[0], R1 = R[1], R2 = R[2], R3 = R[3], R4 = R[4], R5 = R[5], R6 = R[6], R7 = R[7], R8 = R[8];
    e[0] = v.a.x - d[0];
    e[1] = v.a.y - d[1];
    e[2] = v.a.z - d[2];
    // R C_A (C_A symmetric: c00 c01 c02 / c11 c12 / c22)
    const float a00 = A.w, a01 = B.x, a02 = B.y, a11 = B.z, a12 = B.w, a22 = C22;
    const float T00 = R0 * a00 + R1 * a01 + R2 * a02, T01 = R0 * a01 + R1 * a11 + R2 * a12,
                T02 = R0 * a02 + R1 * a12 + R2 * a22;
    const float T10 = R3 * a00 + R4 * a01 + R5 * a02, T11 = R3 * a01 + R4 * a11 + R5 * a12,
                T12 = R3 * a02 + R4 * a12 + R5 * a22;
    const float T20 = R6 * a00 + R7 * a01 + R8 * a02, T21 = R6 * a01 + R7 * a11 + R8 * a12,
                T22 = R6 * a02 + R7 * a12 + R8 * a22;
    // M = C_B + (R C_A) R^T
    const float m00 = v.a.w + T00 * R0 + T01 * R1 + T02 * R2;
    const float m01 = v.b.x + T00 * R3 + T01 * R4 + T02 * R5;
    const float m02 = v.b.y + T00 * R6 + T01 * R7 + T02 * R8;
    const float m11 = v.b.z + T10 * R3 + T11 * R4 + T12 * R5;
    const float m12 = v.b.w + T10 * R6 + T11 * R7 + T12 * R8;
    const float m22 = v.c.x + T20 * R6 + T21 * R7 + T22 * R8;
    // Omega = M^-1 by the adjugate
    const float c00 = m11 * m22 - m12 * m12, c01 = m02 * m12 - m01 * m22, c02 = m01 * m12 - m02 * m11;
    const float c11 = m00 * m22 - m02 * m02, c12 = m01 * m02 - m00 * m12, c22 = m00 * m11 - m01 * m01;
    const float det = m00 * c00 + m01 * c01 + m02 * c02;
    if (!(det > 0.f)) return false;
    const float id = __frcp_rn(det);
    o[0] = c00 * id;
    o[1] = c01 * id;
    o[2] = c02 * id;
    o[3] = c11 * id;
    o[4] = c12 * id;
    o[5] = c22 * id;
    w[0] = o[0] * e[0] + o[1] * e[1] + o[2] * e[2];
    w[1] = o[1] * e[0] + o[3] * e[1] + o[4] * e[2];
    w[2] = o[2] * e[0] + o[4] * e[1] + o[5] * e[2];
    return true;
}

// One correspondence's cost e' Omega e (Eq. 2) added to acc[0] (error evaluation).
__device__ __forceinline__ int accumulate_cost(float acc[1], const float *R, const float4 &A, const float4 &B,
                                               float C22, const VoxelRec &v, const float d[3])
{
    float e[3], o[6], w[3];
    if (!point_omega(R, A, B, C22, v, d, e, o, w)) return 0;
    acc[0] += e[0] * w[0] + e[1] * w[1] + e[2] * w[2];
    return 1;
}

// One correspondence's contribution (Eq. 2, 5, 6 in the adjoint form) added to acc.
__device__ __forceinline__ void accumulate_terms(float acc[kNT], const float e[3], const float o[6], const float w[3],
                                                 const float x[3])
{
    const float e0 = e[0], e1 = e[1], e2 = e[2];
    const float o00 = o[0], o01 = o[1], o02 = o[2], o11 = o[3], o12 = o[4], o22 = o[5];
    const float w0 = w[0], w1 = w[1], w2 = w[2];
    const float x0 = x[0], x1 = x[1], x2 = x[2];   // lever arm a = R p
    // P = [a]x Omega  (= H_wv contribution)
    const float P00 = x1 * o02 - x2 * o01, P01 = x1 * o12 - x2 * o11, P02 = x1 * o22 - x2 * o12;
    const float P10 = x2 * o00 - x0 * o02, P11 = x2 * o01 - x0 * o12, P12 = x2 * o02 - x0 * o22;
    const float P20 = x0 * o01 - x1 * o00, P21 = x0 * o11 - x1 * o01, P22 = x0 * o12 - x1 * o02;
    // H_ww = -[a]x Omega [a]x = -P [a]x (upper triangle)
    acc[0] += P02 * x1 - P01 * x2;
    acc[1] += P00 * x2 - P02 * x0;
    acc[2] += P01 * x0 - P00 * x1;
    acc[3] += P10 * x2 - P12 * x0;
    acc[4] += P11 * x0 - P10 * x1;
    acc[5] += P21 * x0 - P20 * x1;
    acc[6] += P00; acc[7] += P01; acc[8] += P02;
    acc[9] += P10; acc[10] += P11; acc[11] += P12;
    acc[12] += P20; acc[13] += P21; acc[14] += P22;
    acc[15] += o00; acc[16] += o01; acc[17] += o02; acc[18] += o11; acc[19] += o12; acc[20] += o22;
    // b_w = a x w, b_v = w
    acc[21] += x1 * w2 - x2 * w1;
    acc[22] += x2 * w0 - x0 * w2;
    acc[23] += x0 * w1 - x1 * w0;
    acc[24] += w0; acc[25] += w1; acc[26] += w2;
    acc[27] += e0 * w0 + e1 * w1 + e2 * w2;
}

__device__ __forceinline__ int accumulate_point(float acc[kNT], const float *R, const float4 &A, const float4 &B,
                                                float C22, const VoxelRec &v, const float d[3], const float x[3])
{
    float e[3], o[6], w[3];
    if (!point_omega(R, A, B, C22, v, d, e, o, w)) return 0;
    accumulate_terms(acc, e, o, w, x);
    return 1;
}

template <int NT>
__device__ __forceinline__ int accumulate(float acc[NT], const float *R, const float4 &A, const float4 &B, float C22,
                                          const VoxelRec &v, const float d[3], const float x[3])
{
    if constexpr (NT == 1)
        return accumulate_cost(acc, R, A, B, C22, v, d);
    else
        return accumulate_point(acc, R, A, B, C22, v, d, x);
}

// A correspondence weighted by wgt (the voxel's point count): Omega scaled.
template <int NT>
__device__ __forceinline__ int accumulate_weighted(float acc[NT], const float *R, const float4 &A, const float4 &B,
                                                   float C22, const VoxelRec &v, const float d[3], const float x[3],
                                                   float wgt)
{
    float e[3], o[6], w[3];
    if (!point_omega(R, A, B, C22, v, d, e, o, w)) return 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) o[j] *= wgt;
#pragma unroll
    for (int j = 0; j < 3; ++j) w[j] *= wgt;
    if constexpr (NT == 1)
        acc[0] += e[0] * w[0] + e[1] * w[1] + e[2] * w[2];
    else
        accumulate_terms(acc, e, o, w, x);
    return 1;
}

// Voxel offsets searched around a point's own voxel for the neighbour
// association: the own voxel, the six face neighbours (-x, +x, -y, +y, -z, +z),
// then the twenty other voxels of the 3x3x3 block, x outermost, each coordinate
// running -1, 0, 1.  The first 1, 7 or 27 entries are used.
__constant__ int8_t c_nb_off[27][3] = {
    {0, 0, 0},   {-1, 0, 0},  {1, 0, 0},   {0, -1, 0},  {0, 1, 0},   {0, 0, -1},  {0, 0, 1},
    {-1, -1, -1}, {-1, -1, 0}, {-1, -1, 1}, {-1, 0, -1}, {-1, 0, 1},  {-1, 1, -1}, {-1, 1, 0},
    {-1, 1, 1},  {0, -1, -1}, {0, -1, 1},  {0, 1, -1},  {0, 1, 1},   {1, -1, -1}, {1, -1, 0},
    {1, -1, 1},  {1, 0, -1},  {1, 0, 1},   {1, 1, -1},  {1, 1, 0},   {1, 1, 1}};

// Points of one work item for the variants: every voxel of the neighbour set
// around the point's own voxel is a correspondence (e = mu_v - q, the point's
// offset taken relative to that voxel's corner), optionally weighted by the
// voxel's point count.  One point per lane per step, plain loads.
template <int NT, bool FF, bool REC>
__device__ __forceinline__ void linearize_points_general(const PoseParam &P, const MapDesc &m, const FrameDesc &F,
                                                         const WorkItem &w, int lane, float acc[NT], int &inl,
                                                         int nb, int weighted, const CorrRecord &rc, int64_t rbase)
{
    const float4 *__restrict__ pa = F.pa + w.start;
    const float4 *__restrict__ pb = F.pb + w.start;
    const float *__restrict__ pc = F.pc + w.start;
    for (int i = lane; i < w.count; i += 32) {
        const float4 A = __ldg(pa + i), B = __ldg(pb + i);
        const float C = __ldg(pc + i);
        int k[3];
        float d[3], x[3];
        const bool ok = FF ? point_key_ff(P, m, A.x, A.y, A.z, k, d, x) : point_key_split(P, m, A.x, A.y, A.z, k, d, x);
        if (!ok) {
            record_point<REC>(rc, rbase + i, false, 0ull, 0);
            continue;
        }
        int32_t found = 0;
        for (int j = 0; j < nb; ++j) {
            int kk[3];
            bool in = true;
            float dj[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int o = c_nb_off[j][a];
                kk[a] = k[a] + o;
                in = in && kk[a] >= -kKeyOffset && kk[a] <= kKeyOffset - 1;
                dj[a] = __fmaf_rn(-(float)o, m.r_l, __fmaf_rn(-(float)o, m.r_h, d[a]));
            }
            if (!in) continue;
            const int slot = probe(m.keys, m.mask, m.log2cap, pack_key(kk[0], kk[1], kk[2]));
            if (slot < 0) continue;
            found |= 1 << j;
            const VoxelRec v = m.rec[slot];
            const float wgt = weighted ? (float)__float_as_uint(v.c.y) : 1.f;
            inl += accumulate_weighted<NT>(acc, P.Rh, A, B, C, v, dj, x, wgt);
        }
        record_point<REC>(rc, rbase + i, true, pack_key(k[0], k[1], k[2]), found);
    }
}

// Work items belong to single warps: a warp copies its factor's parameters to
// its own shared-memory slot, runs over the item's points, reduces its 28 sums
// by shuffles and writes them as float64 -- no block barriers anywhere.  Warps
// take items in list order from a global counter.
// Live groups (kGroup consecutive points) gw .. gw + 31 of a work item, one bit
// each: every group in range when the pair has no group test, else those whose
// box may reach a voxel of the target (group_live; a dead group provably has no
// correspondence).  The item starts on a group boundary.
template <class L>
__device__ __forceinline__ uint32_t live_groups(const PoseParam &P, const MapDesc &m, const FrameDesc &F,
                                                const WorkItem &w, int gw, int ng, int lane)
{
    if (P.cs < 0) return (ng - gw >= 32) ? 0xffffffffu : ((1u << (ng - gw)) - 1u);
    const bool l = gw + lane < ng &&
                   group_live<L>(P, F.gbox + 6 * ((w.start >> 5) + gw + lane), m.r_h, m.inv_rf, m.coarse);
    return __ballot_sync(0xffffffffu, l);
}

// Points of one work item, one lane per point.  The item's groups are taken in
// runs of consecutive live groups (all of them when the pair has no group
// test); dead groups are never visited.  Each lane adds its points in index
// order whether or not dead groups are skipped, so the sums do not change.
//   PTS = 1: one point per lane per step, the next step's point loads issued
//            before this step's key, probe and record chain;
//   PTS = 2: two points per lane per step, both points' loads, keys and first
//            probes issued before either record is needed.
template <int PTS, bool FF, int NT, bool REC = false, class L = LdNC>
__device__ __forceinline__ void linearize_points(const PoseParam &P, const MapDesc &m, const FrameDesc &F,
                                                 const WorkItem &w, int lane, float acc[NT], int &inl,
                                                 const CorrRecord &rc = CorrRecord{}, int64_t rbase = 0)
{
    const float4 *__restrict__ pa = F.pa + w.start;
    const float4 *__restrict__ pb = F.pb + w.start;
    const float *__restrict__ pc = F.pc + w.start;
    const int n_all = w.count, ng = (n_all + kGroup - 1) / kGroup;
    for (int gw = 0; gw < ng; gw += 32) {
        uint32_t live = live_groups<L>(P, m, F, w, gw, ng, lane);
        while (live) {
            // the next run of consecutive live groups: points [i_begin, n)
            const int a = __ffs(live) - 1;
            const uint32_t rest = ~(live >> a);
            const int len = rest ? __ffs(rest) - 1 : 32 - a;
            live = (a + len >= 32) ? 0u : (live & (~0u << (a + len)));
            const int i_begin = (gw + a) * kGroup;
            const int n = min(n_all, (gw + a + len) * kGroup);
            if (PTS == 1) {
                float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A;
                float C = 0.f;
                if (i_begin + lane < n) {
                    A = L::ld(pa + i_begin + lane);
                    B = L::ld(pb + i_begin + lane);
                    C = L::ld(pc + i_begin + lane);
                }
                for (int i = i_begin + lane; i < n; i += 32) {
                    const float4 A0 = A, B0 = B;
                    const float C0 = C;
                    if (i + 32 < n) {
                        A = L::ld(pa + i + 32);
                        B = L::ld(pb + i + 32);
                        C = L::ld(pc + i + 32);
                    }
                    float d0[3], x0[3];
                    const PointSlot s0 = point_hash<FF>(P, m, A0.x, A0.y, A0.z, d0, x0);
                    uint64_t f0 = kEmptyKey;
                    VoxelRec v0;
                    if (s0.ok) {   // the record of the first slot probed travels with its key
                        f0 = L::ld(m.keys + s0.h);
                        v0 = load_rec<L>(m.rec + s0.h);
                    }
                    const int slot0 = resolve_slot<L>(m, s0, f0);
                    record_point<REC>(rc, rbase + i, s0.ok, s0.key, slot0 >= 0);
                    if (slot0 < 0) continue;
                    if (slot0 != (int)s0.h) v0 = load_rec<L>(m.rec + slot0);
                    inl += accumulate<NT>(acc, P.Rh, A0, B0, C0, v0, d0, x0);
                }
            } else {
                for (int i0 = i_begin + lane; i0 < n; i0 += 64) {
                    const int i1 = i0 + 32;
                    const bool h1 = i1 < n;
                    const float4 A0 = L::ld(pa + i0), B0 = L::ld(pb + i0);
                    const float C0 = L::ld(pc + i0);
                    float4 A1 = make_float4(0.f, 0.f, 0.f, 0.f), B1 = A1;
                    float C1 = 0.f;
                    if (h1) {
                        A1 = L::ld(pa + i1);
                        B1 = L::ld(pb + i1);
                        C1 = L::ld(pc + i1);
                    }
                    float d0[3], x0[3], d1[3], x1[3];
                    PointSlot s0 = point_hash<FF>(P, m, A0.x, A0.y, A0.z, d0, x0);
                    PointSlot s1 = point_hash<FF>(P, m, A1.x, A1.y, A1.z, d1, x1);
                    s1.ok = s1.ok && h1;
                    uint64_t f0 = kEmptyKey, f1 = kEmptyKey;
                    VoxelRec v0, v1;
                    if (s0.ok) {
                        f0 = L::ld(m.keys + s0.h);
                        v0 = load_rec<L>(m.rec + s0.h);
                    }
                    if (s1.ok) {
                        f1 = L::ld(m.keys + s1.h);
                        v1 = load_rec<L>(m.rec + s1.h);
                    }
                    const int slot0 = resolve_slot<L>(m, s0, f0);
                    const int slot1 = resolve_slot<L>(m, s1, f1);
                    record_point<REC>(rc, rbase + i0, s0.ok, s0.key, slot0 >= 0);
                    if (h1) record_point<REC>(rc, rbase + i1, s1.ok, s1.key, slot1 >= 0);
                    if (slot0 >= 0 && slot0 != (int)s0.h) v0 = load_rec<L>(m.rec + slot0);
                    if (slot1 >= 0 && slot1 != (int)s1.h) v1 = load_rec<L>(m.rec + slot1);
                    if (slot0 >= 0) inl += accumulate<NT>(acc, P.Rh, A0, B0, C0, v0, d0, x0);
                    if (slot1 >= 0) inl += accumulate<NT>(acc, P.Rh, A1, B1, C1, v1, d1, x1);
                }
            }
        }
    }
}

// Asynchronous global -> shared copies (cp.async): data in flight occupy
// shared memory, not registers.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst)), "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// One warp's staging area: a ring of three 32-point steps of source data and a
// double buffer of the first probed slot's key and record, one entry per lane.
struct WarpStage {
    float4 pa[3][32];
    float4 pb[3][32];
    float pc[3][32];
    float4 ra[2][32];
    float4 rb[2][32];
    float rc[2][32];
    unsigned long long key[2][32];
};

// Points of one work item as a software pipeline per lane: step st + 2's point
// data are copied in while step st + 1's voxel key is computed and its first
// probe (key and record together) is copied in, while step st's correspondence
// is resolved and accumulated.  Each lane reads back only the slots it filled,
// and refills a slot only after it consumed the slot's values.
template <bool FF, int NT, bool REC>
__device__ __forceinline__ void linearize_points_staged(const PoseParam &P, const MapDesc &m, const FrameDesc &F,
                                                        const WorkItem &w, int lane, float acc[NT], int &inl,
                                                        WarpStage &S, const CorrRecord &rc, int64_t rbase)
{
    const float4 *__restrict__ pa = F.pa + w.start;
    const float4 *__restrict__ pb = F.pb + w.start;
    const float *__restrict__ pc = F.pc + w.start;
    const int n = w.count, steps = (n + 31) >> 5;
    auto issue_points = [&](int st) {
        const int i = (st << 5) + lane;
        if (st < steps && i < n) {
            const int b = st % 3;
            cp_async16(&S.pa[b][lane], pa + i);
            cp_async16(&S.pb[b][lane], pb + i);
            cp_async4(&S.pc[b][lane], pc + i);
        }
    };
    auto issue_probe = [&](const PointSlot &ps, int b) {
        if (ps.ok) {
            cp_async8(&S.key[b][lane], m.keys + ps.h);
            cp_async16(&S.ra[b][lane], &m.rec[ps.h].a);
            cp_async16(&S.rb[b][lane], &m.rec[ps.h].b);
            cp_async4(&S.rc[b][lane], &m.rec[ps.h].c.x);
        }
    };
    issue_points(0);
    cp_async_commit();
    issue_points(1);
    cp_async_commit();
    cp_async_wait<1>();                               // step 0's points
    PointSlot s;
    float d[3], x[3];
    {
        const float4 A = S.pa[0][lane];
        s = point_hash<FF>(P, m, A.x, A.y, A.z, d, x);
        s.ok = s.ok && lane < n;
        issue_probe(s, 0);
        cp_async_commit();
    }
    for (int st = 0; st < steps; ++st) {
        // in flight: the points of st + 1, then the probe of st
        issue_points(st + 2);
        cp_async_commit();
        cp_async_wait<1>();                           // all but step st + 2's points
        PointSlot s1;
        float d1[3], x1[3];
        s1.ok = false;
        if (st + 1 < steps) {
            const float4 A = S.pa[(st + 1) % 3][lane];
            s1 = point_hash<FF>(P, m, A.x, A.y, A.z, d1, x1);
            s1.ok = s1.ok && ((st + 1) << 5) + lane < n;
            issue_probe(s1, (st + 1) & 1);
        }
        cp_async_commit();
        if constexpr (REC) {
            const int i = (st << 5) + lane;
            if (i < n) record_point<REC>(rc, rbase + i, s.ok, s.key, s.ok && resolve_slot(m, s, S.key[st & 1][lane]) >= 0);
        }
        if (s.ok) {
            const int b = st & 1;
            const int slot = resolve_slot(m, s, S.key[b][lane]);
            if (slot >= 0) {
                VoxelRec v;
                if (slot == (int)s.h) {
                    v.a = S.ra[b][lane];
                    v.b = S.rb[b][lane];
                    v.c = make_float4(S.rc[b][lane], 0.f, 0.f, 0.f);
                } else {
                    v = load_rec(m.rec + slot);
                }
                const int q = st % 3;
                inl += accumulate<NT>(acc, P.Rh, S.pa[q][lane], S.pb[q][lane], S.pc[q][lane], v, d, x);
            }
        }
        s = s1;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            d[a] = d1[a];
            x[a] = x1[a];
        }
    }
    cp_async_wait<0>();
}

// One work item: skipped when every cull chunk it spans is dead (no point of it
// can find a voxel), otherwise all of its points.
template <int PTS, bool FF, int NT, bool REC>
__device__ __forceinline__ void linearize_warp_item(const PoseParam &P, const MapDesc &m, const FrameDesc &F,
                                                    const WorkItem &w, int lane, float acc[NT], int &inl,
                                                    WarpStage *S, int nb, int weighted, const CorrRecord &rc)
{
    if (w.count <= 0) return;
    const int c0 = (int)(w.start >> F.cshift), c1 = (int)((w.start + w.count - 1) >> F.cshift);
    const uint32_t span = (c1 - c0 >= 31) ? 0xffffffffu : (((1u << (c1 - c0 + 1)) - 1u) << c0);
    if ((P.cmask & span) == 0u) return;
    int64_t rbase = 0;
    if constexpr (REC) rbase = rc.base[w.unit] + w.start;
    if (nb > 1 || weighted)
        linearize_points_general<NT, FF, REC>(P, m, F, w, lane, acc, inl, nb, weighted, rc, rbase);
    else if constexpr (PTS == 0)
        linearize_points_staged<FF, NT, REC>(P, m, F, w, lane, acc, inl, *S, rc, rbase);
    else
        linearize_points<PTS, FF, NT, REC>(P, m, F, w, lane, acc, inl, rc, rbase);
}

// ------------------------------------------------ shared-memory map path --
//
// Work units are runs of work items that share a target map (the item list is
// grouped by target).  A CTA takes a unit, copies the map's image (compact-key
// hash table, voxel ids, dense records) into shared memory unless it holds it
// already, and its warps run the unit's items probing shared memory only; maps
// without an image take the global-memory path inside the same unit.  The
// per-point arithmetic and the per-lane order are those of the global path.
constexpr int kImgBlock = 512;

template <bool FF, bool REC>
__device__ __forceinline__ void linearize_points_img(const PoseParam &P, const MapDesc &m, const FrameDesc &F,
                                                     const WorkItem &w, int lane, float acc[kNT], int &inl,
                                                     const uint32_t *__restrict__ hdr, const CorrRecord &rc,
                                                     int64_t rbase)
{
    const uint32_t lg = hdr[1], mask = (1u << lg) - 1u;
    const uint32_t ex = hdr[3] & 0xffffu, ey = hdr[3] >> 16, ez = hdr[7];
    const int kb0 = (int)hdr[4], kb1 = (int)hdr[5], kb2 = (int)hdr[6];
    const uint32_t *__restrict__ keys = hdr + kImgHeader / 4;
    const uint16_t *__restrict__ vids = (const uint16_t *)(keys + (1u << lg));
    const float *__restrict__ recs = (const float *)((const unsigned char *)hdr + kImgHeader + img_table_bytes(lg));
    const float4 *__restrict__ pa = F.pa + w.start;
    const float4 *__restrict__ pb = F.pb + w.start;
    const float *__restrict__ pc = F.pc + w.start;
    const int n = w.count;
    float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A;
    float C = 0.f;
    if (lane < n) {
        A = __ldg(pa + lane);
        B = __ldg(pb + lane);
        C = __ldg(pc + lane);
    }
    for (int i = lane; i < n; i += 32) {
        const float4 A0 = A, B0 = B;
        const float C0 = C;
        if (i + 32 < n) {
            A = __ldg(pa + i + 32);
            B = __ldg(pb + i + 32);
            C = __ldg(pc + i + 32);
        }
        int k[3];
        float d[3], x[3];
        const bool ok = FF ? point_key_ff(P, m, A0.x, A0.y, A0.z, k, d, x)
                           : point_key_split(P, m, A0.x, A0.y, A0.z, k, d, x);
        if (!ok) {
            record_point<REC>(rc, rbase + i, false, 0ull, 0);
            continue;
        }
        const uint32_t dx = (uint32_t)(k[0] - kb0), dy = (uint32_t)(k[1] - kb1), dz = (uint32_t)(k[2] - kb2);
        if (dx > ex || dy > ey || dz > ez) {                  // outside the voxel box: no voxel
            record_point<REC>(rc, rbase + i, true, pack_key(k[0], k[1], k[2]), 0);
            continue;
        }
        const uint32_t ck = pack_compact((int)dx, (int)dy, (int)dz);
        uint32_t h = hash_compact(ck, lg);
        int vid = -1;
        for (uint32_t t = 0; t <= mask; ++t) {
            const uint32_t v = keys[h];
            if (v == ck) {
                vid = vids[h];
                break;
            }
            if (v == kEmptyCompact) break;
            h = (h + 1) & mask;
        }
        record_point<REC>(rc, rbase + i, true, pack_key(k[0], k[1], k[2]), vid >= 0);
        if (vid < 0) continue;
        const float2 *r2 = (const float2 *)(recs + (size_t)vid * kImgRecFloats);
        const float2 q0 = r2[0], q1 = r2[1], q2 = r2[2], q3 = r2[3], q4 = r2[4];
        VoxelRec v;
        v.a = make_float4(q0.x, q0.y, q1.x, q1.y);
        v.b = make_float4(q2.x, q2.y, q3.x, q3.y);
        v.c = make_float4(q4.x, q4.y, 0.f, 0.f);
        inl += accumulate_point(acc, P.Rh, A0, B0, C0, v, d, x);
    }
}

template <bool FF, bool REC>
__global__ void __launch_bounds__(kImgBlock, 1) k_linearize_img(const PoseParam *__restrict__ params,
                                                                const MapDesc *__restrict__ maps,
                                                                const FrameDesc *__restrict__ frames,
                                                                const WorkItem *__restrict__ items,
                                                                const int4 *__restrict__ units, int n_units,
                                                                double *__restrict__ partials,
                                                                int64_t *__restrict__ inl_partials,
                                                                int *__restrict__ next_unit, CorrRecord rc)
{
    extern __shared__ uint4 s_img4[];
    const uint32_t *s_img = (const uint32_t *)s_img4;
    constexpr int NW = kImgBlock / 32;
    constexpr int PW = (int)(sizeof(PoseParam) / 4);
    __shared__ PoseParam sP[NW];
    __shared__ MapDesc sM[NW];
    __shared__ int s_unit, s_map, s_valid;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_map = -1;
    for (;;) {
        __syncthreads();                                // the previous unit's readers are done
        if (threadIdx.x == 0) s_unit = atomicAdd(next_unit, 1);
        __syncthreads();
        const int q = s_unit;
        if (q >= n_units) break;
        const int4 U = units[q];                        // (map, first item, end item, -)
        if (U.x != s_map) {                             // uniform: stage this map's image
            const unsigned char *img = maps[U.x].img;
            const uint32_t valid = __ldg((const uint32_t *)img);
            if (valid) {
                const uint32_t lg = __ldg((const uint32_t *)img + 1), nv = __ldg((const uint32_t *)img + 2);
                const int n4 = (int)(img_bytes((int)lg, (int)nv) / 16);
                const uint4 *src = (const uint4 *)img;
                for (int j = threadIdx.x; j < n4; j += kImgBlock) s_img4[j] = __ldg(src + j);
            }
            if (threadIdx.x == 0) {
                s_map = U.x;
                s_valid = (int)valid;
            }
            __syncthreads();
        }
        const bool staged = s_valid != 0;
        for (int it = U.y + wib; it < U.z; it += NW) {
            const WorkItem w = items[it];
            __syncwarp();
            const uint32_t *src = (const uint32_t *)(params + w.unit);
            uint32_t *dst = (uint32_t *)(sP + wib);
            for (int j = lane; j < PW; j += 32) dst[j] = __ldg(src + j);
            __syncwarp();
            if (lane == 0) sM[wib] = maps[sP[wib].map];
            __syncwarp();
            const PoseParam &P = sP[wib];
            const MapDesc m = sM[wib];
            const FrameDesc F = frames[P.frame];
            float acc[kNT];
#pragma unroll
            for (int j = 0; j < kNT; ++j) acc[j] = 0.f;
            int inl = 0;
            const int c0 = (int)(w.start >> F.cshift), c1 = (int)((w.start + w.count - 1) >> F.cshift);
            const uint32_t span = (c1 - c0 >= 31) ? 0xffffffffu : (((1u << (c1 - c0 + 1)) - 1u) << c0);
            if (w.count > 0 && (P.cmask & span) != 0u) {
                int64_t rbase = 0;
                if constexpr (REC) rbase = rc.base[w.unit] + w.start;
                if (staged)
                    linearize_points_img<FF, REC>(P, m, F, w, lane, acc, inl, s_img, rc, rbase);
                else
                    linearize_points<1, FF, kNT, REC>(P, m, F, w, lane, acc, inl, rc, rbase);
            }
            double mine = 0.0;
#pragma unroll
            for (int j = 0; j < kNT; ++j) {
                float x = acc[j];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == j) mine = (double)x;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) inl += __shfl_xor_sync(0xffffffffu, inl, o);
            if (lane < kNT) partials[(int64_t)it * kNT + lane] = mine;
            if (lane == kNT) inl_partials[it] = inl;
        }
    }
}

template <int BLOCK, int MINB, int PTS, bool FF, int NT = kNT, bool REC = false>
__global__ void __launch_bounds__(BLOCK, MINB) k_linearize_f32(const PoseParam *__restrict__ params,
                                                               const MapDesc *__restrict__ maps,
                                                               const FrameDesc *__restrict__ frames,
                                                               const WorkItem *__restrict__ items, int n_items,
                                                               double *__restrict__ partials,
                                                               int64_t *__restrict__ inl_partials,
                                                               int *__restrict__ next_item, int nb, int weighted,
                                                               CorrRecord rc)
{
    constexpr int NW = BLOCK / 32;
    constexpr int PW = (int)(sizeof(PoseParam) / 4);
    __shared__ PoseParam sP[NW];
    __shared__ MapDesc sM[NW];
    __shared__ WarpStage sS[PTS == 0 ? NW : 1];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (;;) {
        // items in list order, each to the next free warp (uneven items cannot
        // leave SMs idle while one warp finishes a long static share)
        int it = 0;
        if (lane == 0) it = atomicAdd(next_item, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const WorkItem w = items[it];
        __syncwarp();                       // this warp's readers of its slots are done
        const uint32_t *src = (const uint32_t *)(params + w.unit);
        uint32_t *dst = (uint32_t *)(sP + wib);
        for (int j = lane; j < PW; j += 32) dst[j] = __ldg(src + j);
        __syncwarp();
        if (lane == 0) sM[wib] = maps[sP[wib].map];
        __syncwarp();
        const PoseParam &P = sP[wib];
        const MapDesc &m = sM[wib];
        const FrameDesc F = frames[P.frame];
        float acc[NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[j] = 0.f;
        int inl = 0;
        linearize_warp_item<PTS, FF, NT, REC>(P, m, F, w, lane, acc, inl, sS + (PTS == 0 ? wib : 0), nb, weighted,
                                              rc);
        // butterfly: every lane ends with the warp's sums; lane j writes sum j
        // (a cost-only pass takes its sum from the lane that holds the cost in the
        // full pass, so both passes' costs agree bit for bit)
        double mine = 0.0;
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            float x = acc[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == (NT == 1 ? kNT - 1 : j)) mine = (double)x;
        }
        if (NT == 1) mine = __shfl_sync(0xffffffffu, mine, kNT - 1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) inl += __shfl_xor_sync(0xffffffffu, inl, o);
        if (lane < NT) partials[(int64_t)it * NT + lane] = mine;
        if (lane == NT) inl_partials[it] = inl;
    }
}

// Cost-only reduction: each factor's item costs summed in item order (the order
// of the full reduction, so the costs agree bit for bit), and its inliers.
__global__ void k_reduce_cost(const int32_t *__restrict__ item_range, int n_f, const double *__restrict__ partials,
                              const int64_t *__restrict__ inl_p, double *__restrict__ cost,
                              int64_t *__restrict__ inliers)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_f) return;
    const int i0 = item_range[2 * f], i1 = item_range[2 * f + 1];
    double s = 0.0;
    int64_t ni = 0;
    for (int i = i0; i < i1; ++i) {
        s += partials[i];
        ni += inl_p[i];
    }
    cost[f] = s;
    if (inliers) inliers[f] = ni;
}

// One factor's 12x12 system from its summed adjoint-form terms, by one warp:
// lane j < 28 holds sum j, lane 0 the inlier count; H = L H^t L', b = L b^t with
// L = [S' ; -D'] (12 x 6) from the factor's T_BA.  Ht, bt, L, G are the warp's
// scratch (36 + 6 + 72 + 72 doubles, shared memory).  inliers may be null.
__device__ __forceinline__ void finalize_factor(double s, int64_t ni, const double *T, int lane, double *Ht,
                                                double *bt, double *L, double *G, double *Hf, double *bf,
                                                double *cost, int64_t *inliers)
{
    // scatter the 28 sums into H^t (6x6) and b^t
    if (lane < 6) {
        const int ww[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
        Ht[6 * ww[lane][0] + ww[lane][1]] = s;
        Ht[6 * ww[lane][1] + ww[lane][0]] = s;
    } else if (lane < 15) {
        const int r = (lane - 6) / 3, c = (lane - 6) % 3;
        Ht[6 * r + 3 + c] = s;
        Ht[6 * (3 + c) + r] = s;
    } else if (lane < 21) {
        const int vv[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
        const int l = lane - 15;
        Ht[6 * (3 + vv[l][0]) + 3 + vv[l][1]] = s;
        Ht[6 * (3 + vv[l][1]) + 3 + vv[l][0]] = s;
    } else if (lane < 27) {
        bt[lane - 21] = s;
    } else if (lane == 27) {
        *cost = s;
    }
    // L rows 0..5 = S' = [[I, [t]x], [0, I]]; rows 6..11 = -D' = -blkdiag(R', R')
    for (int e = lane; e < 72; e += 32) {
        const int r = e / 6, c = e % 6;
        double v = 0.0;
        if (r < 6) {
            if (r == c) v = 1.0;
            else if (r < 3 && c >= 3) {
                const double tx = T[3], ty = T[7], tz = T[11];
                const double K[3][3] = {{0, -tz, ty}, {tz, 0, -tx}, {-ty, tx, 0}};
                v = K[r][c - 3];
            }
        } else {
            const int rr = r - 6;
            if ((rr < 3) == (c < 3)) v = -T[4 * (c % 3) + (rr % 3)];
        }
        L[e] = v;
    }
    __syncwarp();
    for (int e = lane; e < 72; e += 32) {   // G = L H^t
        const int r = e / 6, c = e % 6;
        double x = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) x += L[6 * r + k] * Ht[6 * k + c];
        G[e] = x;
    }
    __syncwarp();
    for (int e = lane; e < 144; e += 32) {  // H = G L'
        const int r = e / 12, c = e % 12;
        if (c < r) continue;
        double x = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) x += G[6 * r + k] * L[6 * c + k];
        Hf[12 * r + c] = x;
        Hf[12 * c + r] = x;
    }
    if (lane < 12) {
        double x = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) x += L[6 * lane + k] * bt[k];
        bf[lane] = x;
    }
    if (lane == 0 && inliers) *inliers = ni;
    __syncwarp();
}

// One warp per factor: fixed-order float64 sum of the factor's item partials,
// then the 12x12 system (finalize_factor).
__global__ void k_reduce_finalize(const PoseParam *__restrict__ params, const int32_t *__restrict__ item_range,
                                  int n_f, const double *__restrict__ partials, const int64_t *__restrict__ inl_p,
                                  double *__restrict__ H, double *__restrict__ b, double *__restrict__ cost,
                                  int64_t *__restrict__ inliers)
{
    constexpr int WPB = 4;
    __shared__ double sHt[WPB][36], sbt[WPB][6], sL[WPB][72], sG[WPB][72];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int f = blockIdx.x * WPB + warp;
    if (f >= n_f) return;
    const int i0 = item_range[2 * f], i1 = item_range[2 * f + 1];
    double s = 0.0;
    if (lane < kNT)
        for (int i = i0; i < i1; ++i) s += partials[(int64_t)i * kNT + lane];
    int64_t ni = 0;
    if (lane == 0)
        for (int i = i0; i < i1; ++i) ni += inl_p[i];
    finalize_factor(s, ni, params[f].T, lane, sHt[warp], sbt[warp], sL[warp], sG[warp], H + (int64_t)f * 144,
                    b + (int64_t)f * 12, cost + f, inliers ? inliers + f : nullptr);
}

// ------------------------------------------------------------------ f64 ----

constexpr int kF64Block = 64;
constexpr int kF64Terms = 91;   // 78 upper-triangle H, 12 b, 1 cost

__global__ void __launch_bounds__(kF64Block) k_linearize_f64(const PoseParam *__restrict__ prm,
                                                             const MapDesc *__restrict__ maps,
                                                             const FrameDesc *__restrict__ frames, int64_t n,
                                                             double *__restrict__ scratch, unsigned int *ticket,
                                                             double *__restrict__ H, double *__restrict__ b,
                                                             double *__restrict__ cost, int64_t *__restrict__ inliers,
                                                             int nb, int weighted, uint64_t *__restrict__ rec_key,
                                                             int32_t *__restrict__ rec_state)
{
    __shared__ double sT[kF64Terms][kF64Block];
    __shared__ int sInl[kF64Block];
    __shared__ bool amLast;
    const int tid = threadIdx.x;
    const PoseParam P = *prm;
    const MapDesc m = maps[P.map];
    const FrameDesc F = frames[P.frame];
    double run0 = 0.0, run1 = 0.0;
    int inl = 0;
    for (int64_t base = (int64_t)blockIdx.x * kF64Block; base < n; base += (int64_t)gridDim.x * kF64Block) {
        const int64_t i = base + tid;
#pragma unroll
        for (int t = 0; t < kF64Terms; ++t) sT[t][tid] = 0.0;
        if (i < n) {
            const float4 A = F.pa[i], B = F.pb[i];
            const float C22 = F.pc[i];
            int k[3];
            double q[3];
            const bool valid = key_f64(P.T, A.x, A.y, A.z, m.inv_r, k, q);
            int32_t found = 0;
            // correspondences: the containing voxel, or every voxel of the neighbour set
            for (int j = 0; valid && j < nb; ++j) {
                int kk[3];
                bool in = true;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    kk[a] = k[a] + c_nb_off[j][a];
                    in = in && kk[a] >= -kKeyOffset && kk[a] <= kKeyOffset - 1;
                }
                if (!in) continue;
                const int slot = probe(m.keys, m.mask, m.log2cap, pack_key(kk[0], kk[1], kk[2]));
                if (slot < 0) continue;
                found |= 1 << j;
                const VoxelRec v = m.rec[slot];
                double R[3][3], J[3][12], e[3], Om[3][3];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) R[r][c] = P.T[4 * r + c];
                const double CA[3][3] = {{A.w, B.x, B.y}, {B.x, B.z, B.w}, {B.y, B.w, C22}};
                const double CB[3][3] = {{v.a.w, v.b.x, v.b.y}, {v.b.x, v.b.z, v.b.w}, {v.b.y, v.b.w, v.c.x}};
                double RC[3][3], M[3][3];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) RC[r][c] = R[r][0] * CA[0][c] + R[r][1] * CA[1][c] + R[r][2] * CA[2][c];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        M[r][c] = CB[r][c] + RC[r][0] * R[c][0] + RC[r][1] * R[c][1] + RC[r][2] * R[c][2];
                // symmetric inverse by the adjugate (M is symmetric positive definite)
                const double c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1];
                const double c01 = M[0][2] * M[2][1] - M[0][1] * M[2][2];
                const double c02 = M[0][1] * M[1][2] - M[0][2] * M[1][1];
                const double c11 = M[0][0] * M[2][2] - M[0][2] * M[2][0];
                const double c12 = M[0][2] * M[1][0] - M[0][0] * M[1][2];
                const double c22 = M[0][0] * M[1][1] - M[0][1] * M[1][0];
                const double det = M[0][0] * c00 + M[0][1] * c01 + M[0][2] * c02;
                if (!(det > 0.0)) continue;
                const double id = (weighted ? (double)__float_as_uint(v.c.y) : 1.0) / det;
                Om[0][0] = c00 * id; Om[0][1] = c01 * id; Om[0][2] = c02 * id;
                Om[1][0] = c01 * id; Om[1][1] = c11 * id; Om[1][2] = c12 * id;
                Om[2][0] = c02 * id; Om[2][1] = c12 * id; Om[2][2] = c22 * id;
                // mean relative to the voxel corner back to absolute target coordinates
                const double mu[3] = {(double)kk[0] * m.r + (double)v.a.x, (double)kk[1] * m.r + (double)v.a.y,
                                      (double)kk[2] * m.r + (double)v.a.z};
#pragma unroll
                for (int r = 0; r < 3; ++r) e[r] = mu[r] - q[r];
                const double px = A.x, py = A.y, pz = A.z;
                const double Pm[3][3] = {{0, -pz, py}, {pz, 0, -px}, {-py, px, 0}};
                const double Qm[3][3] = {{0, -q[2], q[1]}, {q[2], 0, -q[0]}, {-q[1], q[0], 0}};
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        J[r][c] = -Qm[r][c];
                        J[r][3 + c] = (r == c) ? 1.0 : 0.0;
                        J[r][6 + c] = R[r][0] * Pm[0][c] + R[r][1] * Pm[1][c] + R[r][2] * Pm[2][c];
                        J[r][9 + c] = -R[r][c];
                    }
                ++inl;
                double W[3][12], Oe[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
#pragma unroll
                    for (int c = 0; c < 12; ++c) W[r][c] = Om[r][0] * J[0][c] + Om[r][1] * J[1][c] + Om[r][2] * J[2][c];
                    Oe[r] = Om[r][0] * e[0] + Om[r][1] * e[1] + Om[r][2] * e[2];
                }
                int t = 0;
#pragma unroll
                for (int a = 0; a < 12; ++a)
#pragma unroll
                    for (int c = a; c < 12; ++c) sT[t++][tid] += J[0][a] * W[0][c] + J[1][a] * W[1][c] + J[2][a] * W[2][c];
#pragma unroll
                for (int a = 0; a < 12; ++a) sT[78 + a][tid] += J[0][a] * Oe[0] + J[1][a] * Oe[1] + J[2][a] * Oe[2];
                sT[90][tid] += e[0] * Oe[0] + e[1] * Oe[1] + e[2] * Oe[2];
            }
            if (rec_key) {
                rec_key[i] = valid ? pack_key(k[0], k[1], k[2]) : kEmptyKey;
                rec_state[i] = found;
            }
        }
        __syncthreads();
        for (int c = 0; c < kF64Block; ++c) {
            run0 += sT[tid][c];
            if (tid + kF64Block < kF64Terms) run1 += sT[tid + kF64Block][c];
        }
        __syncthreads();
    }
    // this block's partial
    sInl[tid] = inl;
    __syncthreads();
    double *mine = scratch + (int64_t)blockIdx.x * (kF64Terms + 1);
    mine[tid] = run0;
    if (tid + kF64Block < kF64Terms) mine[tid + kF64Block] = run1;
    if (tid == 0) {
        int64_t s = 0;
        for (int c = 0; c < kF64Block; ++c) s += sInl[c];
        mine[kF64Terms] = (double)s;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) amLast = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!amLast) return;
    __threadfence();
    // last block: fixed-order sum over blocks
    for (int t = tid; t <= kF64Terms; t += kF64Block) {
        double s = 0.0;
        for (int q = 0; q < (int)gridDim.x; ++q) s += __ldcg(scratch + (int64_t)q * (kF64Terms + 1) + t);
        if (t < 78) {
            // upper-triangle index t -> (a, c)
            int a = 0, rem = t;
            while (rem >= 12 - a) { rem -= 12 - a; ++a; }
            const int c = a + rem;
            H[12 * a + c] = s;
            H[12 * c + a] = s;
        } else if (t < 90) {
            b[t - 78] = s;
        } else if (t == 90) {
            *cost = s;
        } else if (inliers) {
            *inliers = (int64_t)s;
        }
    }
    if (tid == 0) *ticket = 0u;
}

// ------------------------------------------------- device request loop ----

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_sys(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_sys32(const int *p)
{
    int v;
    asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned int *p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Copy n 32-bit words from global memory (L2, never a stale L1 line) to dst, by one warp.
__device__ __forceinline__ void warp_copy_cg(uint32_t *dst, const uint32_t *src, int n, int lane)
{
    for (int j = lane; j < n; j += 32) dst[j] = __ldcg(src + j);
}

constexpr int kReqWords = (int)(sizeof(LoopRequest) / 8);
static_assert(sizeof(LoopRequest) % 8 == 0, "request words");

// The dispatcher (warp 0 of block 0): requests in order, each prepared and its
// chunks appended to the work queue, until none arrives for idle_ns or the
// host asks it to stop.  Lane 0 polls the ring (acquire loads at system scope)
// and the warp reads a request only after lane 0 has seen it and the warp has
// synchronised.
__device__ void loop_dispatch(const LoopArgs &a, unsigned long long *sreq, int32_t *skbox, float *sstats,
                              float *scbox)
{
    const int lane = threadIdx.x & 31;
    unsigned long long r = a.ctl->next_req;
    unsigned int tail = a.ctl->item_tail;
    unsigned long long t_last = globaltimer_ns();
    int stop = 0;
    for (;;) {
        const int s = (int)(r % (unsigned long long)a.slots);
        const LoopRequest *q = a.req + s;
        // 0 wait, 1 request r is there, 2 it is there but already answered (a
        // relaunch after an earlier loop ended), 3 idle limit, 4 stop
        int what = 0;
        if (lane == 0) {
            unsigned int ns = 32;
            while (what == 0) {
                if (ld_acquire_sys(&q->seq) == r + 1)
                    what = ld_relaxed_sys(&a.res[s].done) == r + 1 ? 2 : 1;
                else if (ld_relaxed_sys32(&a.exit->stop) != 0)
                    what = 4;
                else if (globaltimer_ns() - t_last > a.idle_ns)
                    what = 3;
                else {
                    __nanosleep(ns);
                    if (ns < 512) ns <<= 1;
                }
            }
        }
        what = __shfl_sync(0xffffffffu, what, 0);
        __syncwarp();
        if (what >= 3) {
            stop = what == 4;
            break;
        }
        if (what == 2) {
            ++r;
            t_last = globaltimer_ns();
            continue;
        }
        const unsigned long long *qw = (const unsigned long long *)q;
        for (int j = lane; j < kReqWords; j += 32) sreq[j] = ld_relaxed_sys(qw + j);
        __syncwarp();
        const LoopRequest &R = *(const LoopRequest *)sreq;
        // the map's voxel box and the frame's statistics and chunk boxes, read
        // from L2 into shared memory for the pose parameters
        warp_copy_cg((uint32_t *)skbox, (const uint32_t *)R.map.kbox, 6, lane);
        warp_copy_cg((uint32_t *)(skbox + 8), (const uint32_t *)R.map.cmeta, 8, lane);
        warp_copy_cg((uint32_t *)sstats, (const uint32_t *)R.frame.stats, kStatCount, lane);
        warp_copy_cg((uint32_t *)scbox, (const uint32_t *)R.frame.cbox, 6 * min(R.frame.nchunks, kMaxCullChunks),
                     lane);
        __syncwarp();
        if (lane == 0) {
            MapDesc m = R.map;
            FrameDesc f = R.frame;
            m.kbox = skbox;
            m.cmeta = skbox + 8;
            f.stats = sstats;
            f.cbox = scbox;
            PoseParam P;
#pragma unroll
            for (int i = 0; i < 12; ++i) P.T[i] = R.T[i];
            split_pose(P.T, P);
            P.map = 0;
            P.frame = 0;
            finish_param(P, m, f, R.cull);
            LoopSlotState &S = a.state[s];
            S.P = P;
            S.map = R.map;
            S.frame = R.frame;
            const int ni = min(max(R.n_items, 0), kLoopMaxItems);
            S.kind = R.kind;
            S.n_items = ni;
            S.chunk = R.chunk;
            S.done_items = 0u;
            S.seq = r + 1;
            for (int k = 0; k < ni; ++k) a.queue[(tail + (unsigned)k) & (a.qcap - 1u)] = make_int2(s, k);
            tail += (unsigned)ni;
            __threadfence();
            st_release_gpu(&a.ctl->item_tail, tail);
        }
        __syncwarp();
        ++r;
        t_last = globaltimer_ns();
    }
    if (lane == 0) {
        st_release_gpu(&a.ctl->quit, 1u);
        a.exit->next_req = r;
        a.exit->status = stop ? (int)VGICP_OK : (int)VGICP_ERR_TIMEOUT;
        __threadfence_system();
    }
}

// A worker warp: chunks from the queue until the dispatcher has ended and no
// chunk is left (or worker_ns pass without either).
__device__ void loop_work(const LoopArgs &a, PoseParam &sP, MapDesc &sM, FrameDesc &sF, double *fin)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned int i = 0;
        if (lane == 0) i = atomicAdd(&a.ctl->item_head, 1u);
        i = __shfl_sync(0xffffffffu, i, 0);
        int go = 0;
        if (lane == 0) {
            const unsigned long long t0 = globaltimer_ns();
            unsigned int ns = 32;
            for (;;) {
                if ((int)(ld_acquire_gpu(&a.ctl->item_tail) - i) > 0) {
                    go = 1;
                    break;
                }
                if (ld_acquire_gpu(&a.ctl->quit)) {
                    go = (int)(ld_acquire_gpu(&a.ctl->item_tail) - i) > 0;
                    break;
                }
                if (globaltimer_ns() - t0 > a.worker_ns) {
                    atomicExch(&a.ctl->status, (unsigned int)VGICP_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(ns);
                if (ns < 1024) ns <<= 1;
            }
        }
        go = __shfl_sync(0xffffffffu, go, 0);
        __syncwarp();
        if (!go) return;
        const int2 e = __ldcg(a.queue + (i & (a.qcap - 1u)));
        LoopSlotState &S = a.state[e.x];
        __syncwarp();
        warp_copy_cg((uint32_t *)&sP, (const uint32_t *)&S.P, (int)(sizeof(PoseParam) / 4), lane);
        warp_copy_cg((uint32_t *)&sM, (const uint32_t *)&S.map, (int)(sizeof(MapDesc) / 4), lane);
        warp_copy_cg((uint32_t *)&sF, (const uint32_t *)&S.frame, (int)(sizeof(FrameDesc) / 4), lane);
        const int kind = __ldcg(&S.kind), n_items = __ldcg(&S.n_items), chunk = __ldcg(&S.chunk);
        const unsigned long long seq = __ldcg(&S.seq);
        __syncwarp();
        const PoseParam &P = sP;
        const MapDesc &m = sM;
        const FrameDesc &F = sF;
        WorkItem w;
        w.unit = e.x;
        w.start = (int64_t)e.y * chunk;
        w.count = (int32_t)min((int64_t)chunk, F.n - w.start);
        const int c0 = (int)(w.start >> F.cshift), c1 = (int)((w.start + w.count - 1) >> F.cshift);
        const uint32_t span = (c1 - c0 >= 31) ? 0xffffffffu : (((1u << (c1 - c0 + 1)) - 1u) << c0);
        const bool live = w.count > 0 && (P.cmask & span) != 0u;
        const int64_t slot_base = (int64_t)e.x * kLoopMaxItems;
        if (kind == kLoopLinearize) {
            float acc[kNT];
#pragma unroll
            for (int j = 0; j < kNT; ++j) acc[j] = 0.f;
            int inl = 0;
            if (live) linearize_points<1, false, kNT, false, LdCG>(P, m, F, w, lane, acc, inl);
            double mine = 0.0;
#pragma unroll
            for (int j = 0; j < kNT; ++j) {
                float x = acc[j];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == j) mine = (double)x;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) inl += __shfl_xor_sync(0xffffffffu, inl, o);
            if (lane < kNT) a.partials[(slot_base + e.y) * kNT + lane] = mine;
            if (lane == kNT) a.counts[slot_base + e.y] = inl;
        } else {
            int hits = 0;
            if (live) {
                const float4 *__restrict__ pa = F.pa + w.start;
                for (int j = lane; j < w.count; j += 32) {
                    const float4 A = __ldcg(pa + j);
                    int k[3];
                    float d[3], x[3];
                    if (point_key_split(P, m, A.x, A.y, A.z, k, d, x) &&
                        probe<LdCG>(m.keys, m.mask, m.log2cap, pack_key(k[0], k[1], k[2])) >= 0)
                        ++hits;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) hits += __shfl_xor_sync(0xffffffffu, hits, o);
            if (lane == 0) a.counts[slot_base + e.y] = hits;
        }
        __threadfence();
        unsigned int prev = 0;
        if (lane == 0) prev = atomicAdd(&S.done_items, 1u);
        prev = __shfl_sync(0xffffffffu, prev, 0);
        if (prev + 1u != (unsigned int)n_items) continue;
        // the request's last chunk: its sums in chunk order, then the result
        __threadfence();
        LoopResult *res = a.res + e.x;
        if (kind == kLoopLinearize) {
            double s = 0.0;
            if (lane < kNT)
                for (int k = 0; k < n_items; ++k) s += __ldcg(a.partials + (slot_base + k) * kNT + lane);
            int64_t ni = 0;
            if (lane == 0)
                for (int k = 0; k < n_items; ++k) ni += __ldcg(a.counts + slot_base + k);
            finalize_factor(s, ni, P.T, lane, fin, fin + 36, fin + 42, fin + 114, res->H, res->b, &res->cost,
                            (int64_t *)&res->count);
        } else if (lane == 0) {
            long long c = 0;
            for (int k = 0; k < n_items; ++k) c += __ldcg(a.counts + slot_base + k);
            res->count = c;
        }
        __threadfence_system();
        __syncwarp();
        if (lane == 0) st_release_sys(&res->done, seq);
    }
}

__global__ void __launch_bounds__(kLoopBlock) k_request_loop(LoopArgs a)
{
    constexpr int NW = kLoopBlock / 32;
    __shared__ PoseParam sP[NW];
    __shared__ MapDesc sM[NW];
    __shared__ FrameDesc sF[NW];
    __shared__ double sFin[NW][186];
    __shared__ __align__(16) unsigned long long sReq[kReqWords];
    __shared__ int32_t sKbox[16];        // voxel box (6), then the map's metadata words (8)
    __shared__ float sStats[kStatCount];
    __shared__ float sCbox[6 * kMaxCullChunks];
    const int wib = threadIdx.x >> 5;
    if (blockIdx.x == 0 && wib == 0) {
        loop_dispatch(a, sReq, sKbox, sStats, sCbox);
        return;
    }
    loop_work(a, sP[wib], sM[wib], sF[wib], sFin[wib]);
}

}  // namespace

void launch_prepare_factors(const int32_t *factor_idx, int n_f, const double *poses, const MapDesc *maps,
                            const FrameDesc *frames, int cull, PoseParam *out, cudaStream_t st)
{
    if (n_f <= 0) return;
    k_prepare_factors<<<(n_f + 127) / 128, 128, 0, st>>>(factor_idx, n_f, poses, maps, frames, cull, out);
}

void launch_prepare_list(const double *T, const int32_t *map_idx, const int32_t *frame_idx, int n,
                         const MapDesc *maps, const FrameDesc *frames, int cull, PoseParam *out, cudaStream_t st)
{
    if (n <= 0) return;
    k_prepare_list<<<(n + 127) / 128, 128, 0, st>>>(T, map_idx, frame_idx, n, maps, frames, cull, out);
}

void launch_prepare_given(const double *T, int map, int frame, const MapDesc *maps, const FrameDesc *frames,
                          int cull, PoseParam *out, cudaStream_t st)
{
    k_prepare_given<<<1, 1, 0, st>>>(T, map, frame, maps, frames, cull, out);
}

void launch_prepare_pairs(const double *poses_src, const double *poses_tgt, const int32_t *frame_idx,
                          const int32_t *map_idx, int n_src, int n_tgt, const MapDesc *maps,
                          const FrameDesc *frames, int cull, PoseParam *out, cudaStream_t st)
{
    const int64_t n = (int64_t)n_src * n_tgt;
    if (n <= 0) return;
    k_prepare_pairs<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(poses_src, poses_tgt, frame_idx, map_idx, n_src,
                                                               n_tgt, maps, frames, cull, out);
}

// Variants of the batched kernel: (points per lane per step, blocks per SM the
// register budget is set for).  Work items are per warp, so the block size only
// sets the occupancy granularity.
template <bool FF, int NT, bool REC = false>
void launch_variant(const PoseParam *params, const MapDesc *maps, const FrameDesc *frames, const WorkItem *items,
                    int n_items, double *partials, int64_t *inl_partials, int *next_item, int variant,
                    int grid_per_sm, int num_sms, int nb, int weighted, cudaStream_t st, CorrRecord rc = CorrRecord{})
{
    switch (variant) {
    case 1: {   // one point per step + prefetch, 128-thread blocks, 6 per SM
        const int g = num_sms * (grid_per_sm > 0 ? grid_per_sm : 6);
        k_linearize_f32<128, 6, 1, FF, NT, REC><<<g, 128, 0, st>>>(params, maps, frames, items, n_items,
                                                                partials, inl_partials, next_item, nb, weighted, rc);
        break;
    }
    case 2: {   // two points per step, 128-thread blocks, 4 per SM
        const int g = num_sms * (grid_per_sm > 0 ? grid_per_sm : 4);
        k_linearize_f32<128, 4, 2, FF, NT, REC><<<g, 128, 0, st>>>(params, maps, frames, items, n_items,
                                                                partials, inl_partials, next_item, nb, weighted, rc);
        break;
    }
    case 3: {   // one point per step + prefetch, 128-thread blocks, 4 per SM (no register cap below 128)
        const int g = num_sms * (grid_per_sm > 0 ? grid_per_sm : 4);
        k_linearize_f32<128, 4, 1, FF, NT, REC><<<g, 128, 0, st>>>(params, maps, frames, items, n_items,
                                                                partials, inl_partials, next_item, nb, weighted, rc);
        break;
    }
    case 4: {   // cp.async pipeline (points two steps, probes one step ahead), 128-thread blocks, 5 per SM
        const int g = num_sms * (grid_per_sm > 0 ? grid_per_sm : 5);
        k_linearize_f32<128, 5, 0, FF, NT, REC><<<g, 128, 0, st>>>(params, maps, frames, items, n_items,
                                                                partials, inl_partials, next_item, nb, weighted, rc);
        break;
    }
    case 5: {   // cp.async pipeline, 128-thread blocks, 6 per SM
        const int g = num_sms * (grid_per_sm > 0 ? grid_per_sm : 6);
        k_linearize_f32<128, 6, 0, FF, NT, REC><<<g, 128, 0, st>>>(params, maps, frames, items, n_items,
                                                                partials, inl_partials, next_item, nb, weighted, rc);
        break;
    }
    default: {  // one point per step + prefetch, 128-thread blocks, 5 per SM
        const int g = num_sms * (grid_per_sm > 0 ? grid_per_sm : 5);
        k_linearize_f32<128, 5, 1, FF, NT, REC><<<g, 128, 0, st>>>(params, maps, frames, items, n_items,
                                                                partials, inl_partials, next_item, nb, weighted, rc);
        break;
    }
    }
}

void launch_linearize_f32(const PoseParam *params, const MapDesc *maps, const FrameDesc *frames,
                          const WorkItem *items, int n_items, double *partials, int64_t *inl_partials,
                          int *next_item, int variant, int grid_per_sm, int num_sms, bool compensated, int nb,
                          int weighted, cudaStream_t st, CorrRecord rec)
{
    if (n_items <= 0) return;
    cudaMemsetAsync(next_item, 0, sizeof(int), st);
    if (rec.key) {
        if (compensated)
            launch_variant<true, kNT, true>(params, maps, frames, items, n_items, partials, inl_partials, next_item,
                                            variant, grid_per_sm, num_sms, nb, weighted, st, rec);
        else
            launch_variant<false, kNT, true>(params, maps, frames, items, n_items, partials, inl_partials, next_item,
                                             variant, grid_per_sm, num_sms, nb, weighted, st, rec);
    } else if (compensated) {
        launch_variant<true, kNT>(params, maps, frames, items, n_items, partials, inl_partials, next_item, variant,
                                  grid_per_sm, num_sms, nb, weighted, st);
    } else {
        launch_variant<false, kNT>(params, maps, frames, items, n_items, partials, inl_partials, next_item, variant,
                                   grid_per_sm, num_sms, nb, weighted, st);
    }
}

void launch_linearize_img(const PoseParam *params, const MapDesc *maps, const FrameDesc *frames,
                          const WorkItem *items, const int4 *units, int n_units, double *partials,
                          int64_t *inl_partials, int *next_unit, int num_sms, bool compensated, cudaStream_t st,
                          CorrRecord rec)
{
    if (n_units <= 0) return;
    cudaMemsetAsync(next_unit, 0, sizeof(int), st);
    const int smem = (int)kImgMaxBytes;
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        kern<<<num_sms, kImgBlock, smem, st>>>(params, maps, frames, items, units, n_units, partials, inl_partials,
                                               next_unit, rec);
    };
    if (rec.key)
        compensated ? go(k_linearize_img<true, true>) : go(k_linearize_img<false, true>);
    else
        compensated ? go(k_linearize_img<true, false>) : go(k_linearize_img<false, false>);
}

void launch_cost_f32(const PoseParam *params, const MapDesc *maps, const FrameDesc *frames, const WorkItem *items,
                     int n_items, double *partials, int64_t *inl_partials, int *next_item, int variant,
                     int grid_per_sm, int num_sms, bool compensated, int nb, int weighted, cudaStream_t st)
{
    if (n_items <= 0) return;
    cudaMemsetAsync(next_item, 0, sizeof(int), st);
    if (compensated)
        launch_variant<true, 1>(params, maps, frames, items, n_items, partials, inl_partials, next_item, variant,
                                grid_per_sm, num_sms, nb, weighted, st);
    else
        launch_variant<false, 1>(params, maps, frames, items, n_items, partials, inl_partials, next_item, variant,
                                 grid_per_sm, num_sms, nb, weighted, st);
}

void launch_reduce_finalize(const PoseParam *params, const int32_t *item_range, int n_f, const double *partials,
                            const int64_t *inl_partials, double *H, double *b, double *cost, int64_t *inliers,
                            cudaStream_t st)
{
    if (n_f <= 0) return;
    k_reduce_finalize<<<(n_f + 3) / 4, 128, 0, st>>>(params, item_range, n_f, partials, inl_partials, H, b, cost,
                                                    inliers);
}

void launch_reduce_cost(const int32_t *item_range, int n_f, const double *partials, const int64_t *inl_partials,
                        double *cost, int64_t *inliers, cudaStream_t st)
{
    if (n_f <= 0) return;
    k_reduce_cost<<<(n_f + 127) / 128, 128, 0, st>>>(item_range, n_f, partials, inl_partials, cost, inliers);
}

int linearize_f64_block() { return kF64Block; }

void launch_linearize_f64(const PoseParam *param, const MapDesc *maps, const FrameDesc *frames, int64_t n,
                          double *scratch, unsigned int *ticket, double *H, double *b, double *cost,
                          int64_t *inliers, int grid, int nb, int weighted, cudaStream_t st, uint64_t *rec_key,
                          int32_t *rec_state)
{
    k_linearize_f64<<<grid, kF64Block, 0, st>>>(param, maps, frames, n, scratch, ticket, H, b, cost, inliers, nb,
                                                weighted, rec_key, rec_state);
}

void launch_request_loop(const LoopArgs &a, int num_sms, cudaStream_t st)
{
    k_request_loop<<<num_sms, kLoopBlock, 0, st>>>(a);
}

}  // namespace vg
