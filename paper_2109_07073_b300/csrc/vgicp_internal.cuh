// Internal device layouts and helpers of the VGICP library (sm_103a).
//
// Data layout in HBM
//   frame  : three coalesced streams per point, 36 B/pt in total
//              pa[i] = (x, y, z, c00)       float4
//              pb[i] = (c01, c02, c11, c12) float4
//              pc[i] = c22                  float
//   voxelmap: open-addressing hash, capacity a power of two
//              keys[cap]  uint64 packed voxel coordinate (EMPTY = all ones)
//              rec[cap]   48 B record per slot: mean relative to the voxel's
//                         lower corner k*r (so residuals never cancel against
//                         large absolute coordinates), covariance, count
//
// Voxel coordinate (Sec. III-A, voxel data association): the reference
// definition is k = floor(fl64(x * inv_r)) with x = fma(R0,px,fma(R1,py,fma(R2,pz,t)))
// in float64.  B300 has little float64 throughput, so the kernels evaluate x in
// float32 arithmetic with a proven error bound and fall back to that float64
// definition only for the points whose floor the bound cannot decide.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vg {

constexpr uint64_t kEmptyKey = ~0ull;
constexpr int kKeyOffset = 1 << 20;   // 21-bit two's-complement range [-2^20, 2^20 - 1]
constexpr double kKeyMin = -1048576.0;
constexpr double kKeyMax = 1048575.0;

struct __align__(16) VoxelRec {
    float4 a;   // mu_rel.x, mu_rel.y, mu_rel.z, c00
    float4 b;   // c01, c02, c11, c12
    float4 c;   // c22, count (uint32 bits), unused, unused
};

// Shared-memory image of a small voxelmap (at most kImgMaxVoxels voxels, box
// within the compact-key extents), kept in the map's allocation: a 32-byte
// header (valid, lg, nv, -, box minimum x y z, -), a hash table of 2^lg
// box-relative compact keys (load <= 1/2), the voxel id of each slot (uint16),
// and the voxels' records packed densely, kImgRecFloats floats each: mean
// relative to the voxel corner (3), covariance (6), count (uint32 bits).  One
// CTA copies it into shared memory and probes without global-memory gathers.
// It is made on demand: when a linearisation that reads it first runs, and
// again after the map is rebuilt.
// Header words: 0 valid, 1 lg, 2 nv, 3 box extents x | y << 16, 4-6 box
// minimum, 7 box extent z.
constexpr int kImgMaxVoxels = 4096;
constexpr int kImgRecFloats = 10;
constexpr size_t kImgHeader = 32;
__host__ __device__ constexpr size_t img_table_bytes(int lg) { return (size_t)6 << lg; }
__host__ __device__ constexpr size_t img_bytes(int lg, int nv)
{
    return (kImgHeader + img_table_bytes(lg) + (size_t)nv * kImgRecFloats * 4 + 15) & ~(size_t)15;
}
constexpr size_t kImgMaxBytes = img_bytes(13, kImgMaxVoxels);

struct MapDesc {
    uint64_t *keys;
    VoxelRec *rec;
    unsigned char *img;  // shared-memory image (header word 0 = 1 when valid)
    int32_t *kbox;       // device: min voxel coordinate (3), max voxel coordinate (3)
    uint32_t *ckeys;     // compact presence table (capacity cap; the first 2^cmeta[0] entries used)
    int32_t *cmeta;      // device: log2 of the compact table's used capacity, 1 if the map has one
                         // (cmeta[4] coarse shift or -1, cmeta[5..7] coarse grid extents)
    uint32_t *coarse;    // coarse occupancy bitmap over the voxel box (kCoarseWords words)
    uint32_t mask;       // cap - 1
    uint32_t log2cap;    // >= 4
    double r, inv_r;     // resolution and fl64(1 / r)
    float r_h, r_l;      // r = r_h + r_l (float32 pair)
    float inv_rf;        // fl32(inv_r)
    int32_t pow2;        // r is a power of two
};

struct FrameDesc {
    const float4 *pa;
    const float4 *pb;
    const float *pc;
    int64_t n;
    const float *stats;  // device: kStat* entries below
    const float *cbox;   // device: per cull chunk min xyz, max xyz (6 floats; at most kMaxCullChunks)
    int32_t cshift;      // cull chunk = 2^cshift consecutive points (>= 10, so <= 32 chunks)
    int32_t nchunks;
    const int32_t *perm; // device: given index of the point stored at each position (null: given order)
    const float *gbox;   // device: per group of kGroup consecutive points min xyz, max xyz (finite points)
};

// Groups of consecutive stored points with a bounding box each (exact culling
// below the cull chunks: with the points in spatial order a group is compact).
constexpr int kGroup = 32;
// Coarse occupancy of a voxelmap: one bit per cell of 2^shift x 2^shift x 2^shift
// voxels over its voxel box (shift >= 2, the smallest that fits kCoarseWords
// words), set when the cell holds a voxel.  A group test spanning more than
// kCoarseMaxCells cells takes the group as live without looking.
constexpr int kCoarseWords = 1024;
constexpr int kCoarseMaxCells = 16;

constexpr int kMaxCullChunks = 32;

// Points per work item of a factor of n source points: the configured chunk,
// except that a small factor is cut into at least kMinFactorItems items (a
// multiple of 32 points each, at least 64) so that it alone still keeps several
// warps busy.  It depends on the factor's own size only, so a factor's items,
// and its sums, are the same alone and in any batch.
constexpr int kMinFactorItems = 8;
__host__ __device__ inline int item_chunk(int64_t n, int chunk)
{
    int64_t c = (n + kMinFactorItems - 1) / kMinFactorItems;
    c = (c + 31) & ~(int64_t)31;
    if (c < 64) c = 64;
    return (int)(c < chunk ? c : chunk);
}

// Frame statistics, over the points with finite coordinates.
enum {
    kStatCmax = 0,   // max |covariance entry|
    kStatPmax = 1,   // max |x|, |y|, |z| (3)
    kStatMin = 4,    // min x, y, z as order-preserving uint32 (3)
    kStatMax = 7,    // max x, y, z as order-preserving uint32 (3)
    kStatCount = 10
};

// float <-> uint32 mapping that preserves order (for atomicMin / atomicMax)
constexpr uint32_t kOrderedPosInf = 0xFF800000u;   // ordered_bits(+inf)
constexpr uint32_t kOrderedNegInf = 0x007FFFFFu;   // ordered_bits(-inf)
__device__ __forceinline__ uint32_t ordered_bits(float x)
{
    const uint32_t b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_ordered_bits(uint32_t o)
{
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Per-factor (or per-pair) transform in the forms the kernels use.
struct __align__(16) PoseParam {
    double T[12];        // T_BA exactly as defined (float64)
    float Rh[9], Rl[9];  // R = Rh + Rl (float32 pairs), row-major
    float th[3], tl[3];  // t = th + tl
    int32_t map, frame;  // descriptor-table indices
    // split translation t = k0 r + tf for the float32 voxel floor (overlap)
    int32_t k0[3];
    float tfh[3];        // fl32(tf)
    float tol[3];        // float32 floor decided when tol <= x - k r <= rup
    float rup[3];
    // margins of the float32-pair floor (linearisation)
    float ffm[3];        // decided when ffm <= x - k r <= ffup
    float ffup[3];
    int32_t cull;        // 1: the pair provably has no correspondence
    int32_t koff[3];     // target voxel-box minimum minus k0: compact coordinate = floor(x'/r) - koff
    uint32_t cmask;      // bit c: cull chunk c of the source may have correspondences
    float hm[3];         // overlap floor decided when |frac(x / r) - 1/2| <= hm (see axis_box)
    int32_t cs;          // group culling: the target's coarse shift, or -1 (no group test)
    int32_t cext[3];     // coarse grid extents of the target (cells per axis)
    int32_t bext[3];     // voxel box extents of the target minus one (voxels per axis - 1)
};

// ---------------------------------------------------------------- keys ----

// Compact 32-bit voxel key relative to the map's voxel bounding box: 11 bits
// for x and y, 10 for z.  A map has a compact table when its box extent fits
// (x, y <= 2046, z <= 1022), so the all-ones word never names a voxel.
constexpr uint32_t kEmptyCompact = 0xFFFFFFFFu;
constexpr int kCompactMaxX = 2046, kCompactMaxZ = 1022;
// Presence bitmap over a map's voxel box (in place of the compact table when
// it is this small): voxel (dx, dy, dz) relative to the box minimum is bit
// dx + X (dy + Y dz) of the ckeys words, CLEARED when the voxel exists (the
// words start as all ones, like an empty compact table).
constexpr uint32_t kBitmapMaxWords = 32768;

__device__ __forceinline__ uint32_t pack_compact(int dx, int dy, int dz)
{
    return (uint32_t)dx | ((uint32_t)dy << 11) | ((uint32_t)dz << 22);
}

__device__ __forceinline__ uint32_t hash_compact(uint32_t ck, uint32_t log2cap)
{
    return (ck * 0x9E3779B1u) >> (32 - log2cap);
}

__device__ __forceinline__ uint64_t pack_key(int kx, int ky, int kz)
{
    return ((uint64_t)(uint32_t)(kx + kKeyOffset) << 42) | ((uint64_t)(uint32_t)(ky + kKeyOffset) << 21) |
           (uint64_t)(uint32_t)(kz + kKeyOffset);
}

__device__ __forceinline__ void unpack_key(uint64_t key, int &kx, int &ky, int &kz)
{
    kx = (int)((key >> 42) & 0x1FFFFF) - kKeyOffset;
    ky = (int)((key >> 21) & 0x1FFFFF) - kKeyOffset;
    kz = (int)(key & 0x1FFFFF) - kKeyOffset;
}

// Load policies of the gather helpers: the read-only (non-coherent) data path
// for kernels whose inputs cannot change while they run, and L2-only loads for
// the persistent request loop, which reads objects made resident (by other
// kernels, into memory other objects may have used before) after it started.
struct LdNC {
    template <class T>
    __device__ __forceinline__ static T ld(const T *p) { return __ldg(p); }
};
struct LdCG {
    template <class T>
    __device__ __forceinline__ static T ld(const T *p) { return __ldcg(p); }
};

// Multiplicative (Fibonacci) hashing: top log2cap bits of key * 2^64/phi.
__device__ __forceinline__ uint32_t hash_slot(uint64_t key, uint32_t log2cap)
{
    return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - log2cap));
}

// Continue a probe for key from slot s (the caller has checked the slots before).
template <class L = LdNC>
__device__ __forceinline__ int probe_from(const uint64_t *__restrict__ keys, uint32_t mask, uint64_t key, uint32_t s)
{
    for (uint32_t i = 0; i < mask; ++i) {
        const uint64_t k = L::ld(keys + s);
        if (k == key) return (int)s;
        if (k == kEmptyKey) return -1;
        s = (s + 1) & mask;
    }
    return -1;
}

// Slot of key in the map, or -1.  Linear probing; the table always holds an
// empty slot (load <= 2/3), so the loop ends at the first empty slot.
template <class L = LdNC>
__device__ __forceinline__ int probe(const uint64_t *__restrict__ keys, uint32_t mask, uint32_t log2cap,
                                     uint64_t key)
{
    uint32_t s = hash_slot(key, log2cap);
    for (uint32_t i = 0; i <= mask; ++i) {
        const uint64_t k = L::ld(keys + s);
        if (k == key) return (int)s;
        if (k == kEmptyKey) return -1;
        s = (s + 1) & mask;
    }
    return -1;
}

// Reference voxel coordinate in float64: x = fma(R0,px,fma(R1,py,fma(R2,pz,t))),
// k = floor(x * inv_r).  Returns false if any axis is out of range or not finite.
__device__ __forceinline__ bool key_f64(const double *T, float px, float py, float pz, double inv_r,
                                        int k[3], double q[3])
{
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        q[i] = __fma_rn(T[4 * i], (double)px, __fma_rn(T[4 * i + 1], (double)py,
                        __fma_rn(T[4 * i + 2], (double)pz, T[4 * i + 3])));
        const double f = floor(__dmul_rn(q[i], inv_r));
        ok = ok && (f >= kKeyMin && f <= kKeyMax);
        k[i] = ok ? (int)f : 0;
    }
    return ok;
}

// Error-free sum (Knuth): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// x - k*r with r = r_h + r_l, as an unevaluated sum x = s + lo: rounding error
// relative to the result itself (a few float32 ulps of |x - k r|).
__device__ __forceinline__ float face_dist(float s, float lo, float k, float r_h, float r_l)
{
    float g = __fmaf_rn(-k, r_h, s);
    g = __fmaf_rn(-k, r_l, g);
    return __fadd_rn(g, lo);
}

// One axis of the voxel coordinate from a float32-pair transform.
//
// x = Rh.p + th + (Rl.p + tl) is formed as an unevaluated pair (s, lo) with
// error-free products and sums, accurate to ~2^-44 of X = sum |R_j| pmax_j + |t|.
// The float64 reference differs from the exact value by < 2^-50 X (three fmas,
// one multiply by inv_r).  The caller's margins: lo_m = 2^-40 X, and
// up_m = r - lo_m - 2^-22 r (the face distance g0 carries ~2^-24 r of rounding).
// Returns false when x - k r is outside [lo_m, up_m] (or not finite); the caller
// then evaluates the float64 reference.  On success: k is the reference floor
// and d = x - k r in [0, r).
__device__ __forceinline__ bool axis_key_ff(const float *Rh, const float *Rl, float th, float tl, float px,
                                            float py, float pz, float r_h, float r_l, float inv_rf, float lo_m,
                                            float up_m, int &k, float &d, float &rp)
{
    const float h0 = __fmul_rn(Rh[0], px), l0 = __fmaf_rn(Rh[0], px, -h0);
    const float h1 = __fmul_rn(Rh[1], py), l1 = __fmaf_rn(Rh[1], py, -h1);
    const float h2 = __fmul_rn(Rh[2], pz), l2 = __fmaf_rn(Rh[2], pz, -h2);
    float s, e1, e2, e3;
    two_sum(h0, h1, s, e1);
    two_sum(s, h2, s, e2);
    rp = s;                                         // fl32(Rh . p): the lever arm
    two_sum(s, th, s, e3);
    float lo = __fadd_rn(__fadd_rn(l0, l1), __fadd_rn(l2, e1));
    lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(e2, e3), tl));
    lo = __fmaf_rn(Rl[0], px, lo);
    lo = __fmaf_rn(Rl[1], py, lo);
    lo = __fmaf_rn(Rl[2], pz, lo);
    // candidate floor (off by one only within ~2^-24 |x| of a face: then g0 < 0
    // or g0 >= r and the point is left undecided)
    const float kf = floorf(__fmul_rn(__fadd_rn(s, lo), inv_rf));
    const float g0 = face_dist(s, lo, kf, r_h, r_l);
    if (!(g0 >= lo_m && g0 <= up_m)) return false;   // also catches NaN / inf
    if (!(kf >= (float)kKeyMin && kf <= (float)kKeyMax)) {
        k = INT32_MIN;                                // decided: out of range
        return true;
    }
    k = (int)kf;
    d = g0;
    return true;
}

// One axis of the voxel floor from a plain float32 fma chain on the split
// translation: x' = R p + tf with t = k0 r + tf, so floor(x / r) = floor(x' / r) + k0
// and the float32 error bound depends on |R p| + |tf| only, not on |t|.  The
// caller's tol covers the float32 error (2^-22 (sum |R_j| pmax_j + |tf|)), the
// float64 reference's own rounding and the face-distance rounding.  Returns
// false when undecided; k = INT32_MIN marks a decided out-of-range coordinate.
__device__ __forceinline__ bool axis_key_split(const float *Rh, float tfh, float tol, float rup, int k0, float px,
                                               float py, float pz, float r_h, float r_l, float inv_rf, int &k)
{
    const float x = __fmaf_rn(Rh[0], px, __fmaf_rn(Rh[1], py, __fmaf_rn(Rh[2], pz, tfh)));
    const float kf = floorf(__fmul_rn(x, inv_rf));
    const float d = __fmaf_rn(-kf, r_l, __fmaf_rn(-kf, r_h, x));
    if (!(d >= tol && d <= rup)) return false;
    const int kk = (int)kf + k0;
    k = (kk >= -kKeyOffset && kk <= kKeyOffset - 1) ? kk : INT32_MIN;
    return true;
}

// One axis of the floor on the split translation, returned relative to the
// target's voxel box (dx = floor(x / r) - box minimum) for the compact tables:
// coordinates outside the box fail the caller's unsigned range test, so no
// separate validity check is needed.  Returns false when undecided.
__device__ __forceinline__ bool axis_box(const float *Rh, float tfh, float hm, int koff, float px, float py,
                                         float pz, float inv_rf, int &dx)
{
    // y = x / r in float32; its distance to the reference y* = fl64(x64 * fl64(1/r))
    // is below 1/2 - hm (per-pair bound), so floor(y) = floor(y*) when the
    // fraction of y keeps that distance from both faces.  y - floor(y) is exact
    // or rounds towards a face, and so does the 1/2 taken off it.
    const float x = __fmaf_rn(Rh[0], px, __fmaf_rn(Rh[1], py, __fmaf_rn(Rh[2], pz, tfh)));
    const float y = __fmul_rn(x, inv_rf);
    const float kf = floorf(y);
    dx = (int)kf - koff;
    return fabsf(__fsub_rn(__fsub_rn(y, kf), 0.5f)) <= hm;
}

// One axis from a plain float32 fma chain with the error bound
// |x32 - x| <= 2^-20 X (four roundings of at most 2^-24 X each, with margin).
// Returns false when the bound straddles a voxel face.  k = INT32_MIN marks a
// decided out-of-range coordinate.
__device__ __forceinline__ bool axis_key_f32(const float *Rh, float th, float px, float py, float pz, float r_h,
                                             float r_l, float inv_rf, int &k)
{
    const float x = __fmaf_rn(Rh[0], px, __fmaf_rn(Rh[1], py, __fmaf_rn(Rh[2], pz, th)));
    const float X = fabsf(Rh[0] * px) + fabsf(Rh[1] * py) + fabsf(Rh[2] * pz) + fabsf(th);
    const float kf = floorf(__fmul_rn(x, inv_rf));
    const float tol = X * 0x1p-20f + fabsf(kf * r_l) * 2.f + 0x1p-100f;
    const float d0 = __fmaf_rn(-kf, r_h, x);          // ~ x - kf r, error ~ 2^-24 |d0|
    const float d1 = __fmaf_rn(-(kf + 1.f), r_h, x);  // ~ x - (kf+1) r
    if (!(d0 >= tol * 1.0001f && d1 <= -tol * 1.0001f)) return false;
    if (!(kf >= (float)kKeyMin && kf <= (float)kKeyMax)) {
        k = INT32_MIN;
        return true;
    }
    k = (int)kf;
    return true;
}

// Whether a group of source points may have a voxel in the target map under the
// pair's pose; false is exact (no point of the group has one).  gb: the group's
// box (min xyz, max xyz of its finite points; min > max when it has none).  The
// box moves by the float32 pose on the split translation -- centre Rh c + tfh,
// half extent |Rh| h -- grown by 2^-18 of the magnitudes involved plus 1e-6 r:
// 16 times the float32 error of that evaluation and of Rh, tfh against the
// float64 pose, and far above the float64 reference's own rounding.  Divided by
// r with a further 2^-20 relative margin, it gives per axis a range of voxel
// coordinates (relative to the target's voxel box through koff) that holds
// every point's reference coordinate; the coarse cells it spans are looked up in
// the target's coarse occupancy bitmap.  A range outside the box on any axis is
// dead; one spanning more than kCoarseMaxCells cells, or not finite, is live.
template <class L = LdNC>
__device__ __forceinline__ bool group_live(const PoseParam &P, const float *__restrict__ gb, float r_h,
                                          float inv_rf, const uint32_t *__restrict__ coarse)
{
    float b[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) b[j] = L::ld(gb + j);
    if (!(b[0] <= b[3] && b[1] <= b[4] && b[2] <= b[5])) return false;   // no finite point
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float *R = P.Rh + 3 * a;
        float c = P.tfh[a], e = 0.f, mag = fabsf(P.tfh[a]);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float cc = 0.5f * (b[j] + b[3 + j]), hh = 0.5f * (b[3 + j] - b[j]);
            c = fmaf(R[j], cc, c);
            e = fmaf(fabsf(R[j]), hh, e);
            mag = fmaf(fabsf(R[j]), fabsf(cc) + hh, mag);
        }
        const float mu = mag * 0x1p-18f + 1e-6f * r_h + 1e-30f;
        float ylo = (c - e - mu) * inv_rf, yhi = (c + e + mu) * inv_rf;
        const float dy = (fabsf(ylo) + fabsf(yhi)) * 0x1p-20f + 0x1p-20f;
        ylo = floorf(ylo - dy) - (float)P.koff[a];
        yhi = floorf(yhi + dy) - (float)P.koff[a];
        if (yhi < 0.f || ylo > (float)P.bext[a]) return false;       // misses the voxel box
        lo[a] = (int)fmaxf(ylo, 0.f) >> P.cs;                         // (not finite: the whole box)
        hi[a] = (int)fminf(yhi, (float)P.bext[a]) >> P.cs;
    }
    if ((hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1) > kCoarseMaxCells) return true;
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) {
                const uint32_t bit = (uint32_t)x + (uint32_t)P.cext[0] * ((uint32_t)y + (uint32_t)P.cext[1] * (uint32_t)z);
                if ((L::ld(coarse + (bit >> 5)) >> (bit & 31)) & 1u) return true;
            }
    return false;
}

}  // namespace vg
