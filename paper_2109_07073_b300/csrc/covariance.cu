// Per-point covariance from the k nearest neighbours (Sec. III: estimated from
// k neighbouring points once per input cloud), regularised to eigenvalues
// (1, 1, eps) so the surface normal direction receives eps.
//
// Neighbour search on a uniform grid of cell size h:
//   build  cell key per point -> open-addressing table of cells -> per-cell point
//          counts -> exclusive scan -> per-cell point lists;
//   query  cubes of cells around the query grow shell by shell; after shell s
//          every unseen point is at least s*h away, so the search stops once
//          the k-th best squared distance is below (s h)^2.
// Squared distances are formed in float64 as ((dx*dx + dy*dy) + dz*dz), each
// operation separately rounded, and ties go to the lower index, so the
// neighbour set is exactly the one a brute-force scan picks.  The 3x3
// eigen-decomposition is cyclic Jacobi in float64.
#include <algorithm>

#include "kernels.cuh"

namespace vg {

namespace {

constexpr int kMaxK = 32;
constexpr uint32_t kNoCell = 0xFFFFFFFFu;
constexpr int kShellLimit = 12;   // beyond this many shells a query scans every point

__device__ __forceinline__ bool nb_less(double d, int64_t j, double d2, int64_t j2)
{
    return (d < d2) || (d == d2 && j < j2);
}

__device__ __forceinline__ bool finite3(float x, float y, float z)
{
    return isfinite(x) && isfinite(y) && isfinite(z);
}

// cell coordinate of a point, or false when not finite / beyond 2^20 cells
__device__ __forceinline__ bool cell_of(float x, float y, float z, double inv_h, int c[3])
{
    if (!finite3(x, y, z)) return false;
    const double f[3] = {floor((double)x * inv_h), floor((double)y * inv_h), floor((double)z * inv_h)};
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ok = ok && f[i] >= kKeyMin && f[i] <= kKeyMax;
        c[i] = ok ? (int)f[i] : 0;
    }
    return ok;
}

__global__ void k_grid_clear(uint64_t *keys, uint32_t *cnt, uint32_t cap, int *cbox)
{
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += gridDim.x * blockDim.x) {
        keys[s] = kEmptyKey;
        cnt[s] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x < 6) cbox[threadIdx.x] = threadIdx.x < 3 ? INT32_MAX : INT32_MIN;
}

__global__ void k_grid_insert(const float *__restrict__ pts, int64_t n, double inv_h, uint64_t *keys, uint32_t mask,
                              uint32_t lg, uint32_t *cnt, uint32_t *slot_of, int *cbox)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int c[3];
        uint32_t slot = kNoCell;
        if (cell_of(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], inv_h, c)) {
            const uint64_t key = pack_key(c[0], c[1], c[2]);
            uint32_t s = hash_slot(key, lg);
            for (uint32_t t = 0; t <= mask; ++t) {
                const unsigned long long old =
                    atomicCAS((unsigned long long *)(keys + s), (unsigned long long)kEmptyKey, (unsigned long long)key);
                if (old == kEmptyKey || old == key) { slot = s; break; }
                s = (s + 1) & mask;
            }
            if (slot != kNoCell) {
                if (atomicAdd(cnt + slot, 1u) == 0u) {     // first point of a cell: grow the cell box
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        atomicMin(cbox + a, c[a]);
                        atomicMax(cbox + 3 + a, c[a]);
                    }
                }
            }
        }
        slot_of[i] = slot;
    }
}

// exclusive scan of cnt into off (one block; cap is a multiple of its size)
__global__ void k_grid_scan(const uint32_t *__restrict__ cnt, uint32_t *__restrict__ off, uint32_t cap)
{
    __shared__ uint32_t s[1024];
    uint32_t carry = 0;
    for (uint32_t b = 0; b < cap; b += 1024) {
        const uint32_t v = cnt[b + threadIdx.x];
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const uint32_t a = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0u;
            __syncthreads();
            s[threadIdx.x] += a;
            __syncthreads();
        }
        off[b + threadIdx.x] = carry + s[threadIdx.x] - v;
        const uint32_t tot = s[1023];
        __syncthreads();
        carry += tot;
    }
}

__global__ void k_grid_scatter(int64_t n, const uint32_t *__restrict__ slot_of, const uint32_t *__restrict__ off,
                               uint32_t *cur, uint32_t *__restrict__ list)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = slot_of[i];
        if (s == kNoCell) continue;
        list[off[s] + atomicAdd(cur + s, 1u)] = (uint32_t)i;
    }
}

// symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations: A = V diag(w) V'
__device__ void jacobi3(double A[3][3], double w[3], double V[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
    double nrm = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) nrm += A[i][j] * A[i][j];
    nrm = sqrt(nrm);
    for (int sweep = 0; sweep < 64; ++sweep) {
        const double off = sqrt(2.0 * (A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2]));
        if (off <= 1e-15 * nrm || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                const double apq = A[p][q];
                if (apq == 0.0) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
                const double c = rsqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < 3; ++k) {
                    const double x = A[k][p], y = A[k][q];
                    A[k][p] = c * x - s * y;
                    A[k][q] = s * x + c * y;
                }
                for (int k = 0; k < 3; ++k) {
                    const double x = A[p][k], y = A[q][k];
                    A[p][k] = c * x - s * y;
                    A[q][k] = s * x + c * y;
                }
                for (int k = 0; k < 3; ++k) {
                    const double x = V[k][p], y = V[k][q];
                    V[k][p] = c * x - s * y;
                    V[k][q] = s * x + c * y;
                }
            }
    }
    for (int i = 0; i < 3; ++i) w[i] = A[i][i];
}

__global__ void __launch_bounds__(128) k_knn_query(const float *__restrict__ pts, int64_t n, int k, double eps,
                                                   double h, const uint64_t *__restrict__ keys, uint32_t mask,
                                                   uint32_t lg, const uint32_t *__restrict__ cnt,
                                                   const uint32_t *__restrict__ off,
                                                   const uint32_t *__restrict__ list,
                                                   const int *__restrict__ cbox, float *__restrict__ covs)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float qx = pts[3 * i], qy = pts[3 * i + 1], qz = pts[3 * i + 2];
    double bd[kMaxK];
    int64_t bj[kMaxK];
    int cnt_k = 0;
    int c0[3];
    if (cell_of(qx, qy, qz, 1.0 / h, c0)) {
        // shells beyond this one hold no cell of the cloud
        int max_shell = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) max_shell = max(max_shell, max(c0[a] - cbox[a], cbox[3 + a] - c0[a]));
        bool done = false;
        for (int s = 0; s <= min(max_shell, kShellLimit); ++s) {
            // the cells at Chebyshev distance exactly s from c0
            for (int dx = -s; dx <= s; ++dx)
                for (int dy = -s; dy <= s; ++dy) {
                    const bool edge = (dx == -s || dx == s || dy == -s || dy == s);
                    for (int dz = -s; dz <= s; dz += (edge ? 1 : 2 * s)) {
                        const int cx = c0[0] + dx, cy = c0[1] + dy, cz = c0[2] + dz;
                        if (cx < -kKeyOffset || cx >= kKeyOffset || cy < -kKeyOffset || cy >= kKeyOffset ||
                            cz < -kKeyOffset || cz >= kKeyOffset)
                            continue;
                        const int slot = probe(keys, mask, lg, pack_key(cx, cy, cz));
                        if (slot < 0) continue;
                        const uint32_t b = off[slot], e = b + cnt[slot];
                        for (uint32_t t = b; t < e; ++t) {
                            const int64_t j = list[t];
                            const double ddx = __dsub_rn((double)qx, (double)pts[3 * j]);
                            const double ddy = __dsub_rn((double)qy, (double)pts[3 * j + 1]);
                            const double ddz = __dsub_rn((double)qz, (double)pts[3 * j + 2]);
                            const double d =
                                __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
                            if (cnt_k == k && !nb_less(d, j, bd[k - 1], bj[k - 1])) continue;
                            int pos = (cnt_k < k) ? cnt_k++ : k - 1;
                            while (pos > 0 && nb_less(d, j, bd[pos - 1], bj[pos - 1])) {
                                bd[pos] = bd[pos - 1];
                                bj[pos] = bj[pos - 1];
                                --pos;
                            }
                            bd[pos] = d;
                            bj[pos] = j;
                        }
                        if (s == 0) break;   // the single cell of shell 0
                    }
                }
            // every unseen point is at least s*h away
            const double reach = (double)s * h;
            if ((cnt_k == k && bd[k - 1] < reach * reach * (1.0 - 1e-9)) || s == max_shell) {
                done = true;
                break;
            }
        }
        if (!done) {   // sparse neighbourhood: scan every point
            cnt_k = 0;
            for (int64_t j = 0; j < n; ++j) {
                const float x = pts[3 * j], y = pts[3 * j + 1], z = pts[3 * j + 2];
                if (!finite3(x, y, z)) continue;
                const double ddx = __dsub_rn((double)qx, (double)x);
                const double ddy = __dsub_rn((double)qy, (double)y);
                const double ddz = __dsub_rn((double)qz, (double)z);
                const double d = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
                if (cnt_k == k && !nb_less(d, j, bd[k - 1], bj[k - 1])) continue;
                int pos = (cnt_k < k) ? cnt_k++ : k - 1;
                while (pos > 0 && nb_less(d, j, bd[pos - 1], bj[pos - 1])) {
                    bd[pos] = bd[pos - 1];
                    bj[pos] = bj[pos - 1];
                    --pos;
                }
                bd[pos] = d;
                bj[pos] = j;
            }
        }
    }
    float *out = covs + 6 * i;
    if (cnt_k < k) {
        out[0] = 1.f; out[1] = 0.f; out[2] = 0.f; out[3] = 1.f; out[4] = 0.f; out[5] = 1.f;
        return;
    }
    double mean[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < k; ++j)
        for (int a = 0; a < 3; ++a) mean[a] += (double)pts[3 * bj[j] + a];
    for (int a = 0; a < 3; ++a) mean[a] /= (double)k;
    double S[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int j = 0; j < k; ++j) {
        double x[3];
        for (int a = 0; a < 3; ++a) x[a] = (double)pts[3 * bj[j] + a] - mean[a];
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) S[a][c] += x[a] * x[c];
    }
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) S[a][c] /= (double)k;
    double w[3], V[3][3];
    jacobi3(S, w, V);
    // eigenvalues in decreasing order, ties kept in column order
    int o[3] = {0, 1, 2};
    for (int a = 1; a < 3; ++a) {
        const int t = o[a];
        int p = a;
        while (p > 0 && w[o[p - 1]] < w[t]) { o[p] = o[p - 1]; --p; }
        o[p] = t;
    }
    const double lam[3] = {1.0, 1.0, eps};
    double C[3][3];
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int j = 0; j < 3; ++j) s += V[a][o[j]] * lam[j] * V[c][o[j]];
            C[a][c] = s;
        }
    out[0] = (float)C[0][0]; out[1] = (float)C[0][1]; out[2] = (float)C[0][2];
    out[3] = (float)C[1][1]; out[4] = (float)C[1][2]; out[5] = (float)C[2][2];
}

}  // namespace

size_t knn_scratch_bytes(int64_t n)
{
    uint32_t cap = 1024;
    while ((int64_t)cap < 2 * n) cap <<= 1;
    return (size_t)cap * (8 + 4 + 4 + 4) + (size_t)n * 8 + 1024;
}

void launch_knn_covariances(const float *points, int64_t n, int k, double eps, double h, void *scratch, float *covs,
                            cudaStream_t st)
{
    if (n <= 0) return;
    uint32_t cap = 1024, lg = 10;
    while ((int64_t)cap < 2 * n) { cap <<= 1; ++lg; }
    char *p = (char *)scratch;
    uint64_t *keys = (uint64_t *)p;
    uint32_t *cnt = (uint32_t *)(p + (size_t)cap * 8);
    uint32_t *off = cnt + cap;
    uint32_t *cur = off + cap;
    uint32_t *slot_of = cur + cap;
    uint32_t *list = slot_of + n;
    int *cbox = (int *)(list + n);
    const int grid = (int)std::min<int64_t>(148 * 8, (n + 255) / 256);
    k_grid_clear<<<148 * 4, 256, 0, st>>>(keys, cnt, cap, cbox);
    k_grid_insert<<<grid, 256, 0, st>>>(points, n, 1.0 / h, keys, cap - 1, lg, cnt, slot_of, cbox);
    k_grid_scan<<<1, 1024, 0, st>>>(cnt, off, cap);
    cudaMemsetAsync(cur, 0, (size_t)cap * 4, st);
    k_grid_scatter<<<grid, 256, 0, st>>>(n, slot_of, off, cur, list);
    k_knn_query<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(points, n, k, eps, h, keys, cap - 1, lg, cnt, off, list,
                                                            cbox, covs);
}

}  // namespace vg
