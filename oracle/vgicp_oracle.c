/*
 * Plain FP64 CPU oracle for voxelised-GICP factor linearisation, voxelmaps and
 * the voxel overlap metric (Koide et al., "Globally Consistent 3D LiDAR Mapping
 * with GPU-accelerated GICP Matching Cost Factors", RA-L 2021).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA library is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark load it; the CUDA
 * library neither includes nor links it, and it includes nothing of the CUDA
 * library.  Every routine is single-threaded, loops point by point in input
 * order, and accumulates naively in double precision.
 *
 * Conventions (readings of passages the paper leaves open; each is stated in
 * the design notes):
 *   - Poses are 3x4 row-major world-from-frame matrices [R | t] in float64.
 *   - A factor has a target B (owner of the voxelmap) and a source A (whose
 *     points are summed over).  Source points move into the target frame by
 *     T_BA = T_B^-1 T_A (Eq. 3 writes T_ij = T_i^-1 T_j).
 *   - Tangent: right perturbation T <- T Exp(xi), xi = (omega, v), rotation
 *     first; the 12-vector is [xi_B ; xi_A].
 *   - Voxel coordinate of a point (Sec. III-A, voxel data association):
 *     x = fma(R00, px, fma(R01, py, fma(R02, pz, t0))), k = floor(x * inv_r),
 *     inv_r = 1 / r in float64; valid iff -2^20 <= k <= 2^20 - 1 on all axes
 *     (non-finite coordinates are invalid).
 *   - Voxel statistics: mean of the point means and mean of the point
 *     covariances of the points that fall in the voxel (Sec. III-A: VGICP
 *     aggregates point distributions, unlike NDT).
 *   - Covariances are 6 floats (c00, c01, c02, c11, c12, c22).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -o liboracle.so
 * vgicp_oracle.c -lm  (contraction off: every fused multiply-add here is an
 * explicit fma() call).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define KEY_MIN (-1048576.0)   /* -2^20 */
#define KEY_MAX (1048575.0)    /*  2^20 - 1 */

/* ---------------------------------------------------------------- poses -- */

/* T_BA = T_B^-1 T_A with T_B^-1 = [R_B^T | -R_B^T t_B] (Eq. 3, relative pose).
 * R_BA[i][j] = sum_k R_B[k][i] R_A[k][j], t_BA[i] = sum_k R_B[k][i] (t_A[k] - t_B[k]),
 * sums taken k = 0, 1, 2 with separately rounded products. */
void oracle_relative_pose(const double *TB, const double *TA, double *TBA)
{
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s = s + TB[4 * k + i] * TA[4 * k + j];
            TBA[4 * i + j] = s;
        }
        double s = 0.0;
        for (int k = 0; k < 3; ++k) s = s + TB[4 * k + i] * (TA[4 * k + 3] - TB[4 * k + 3]);
        TBA[4 * i + 3] = s;
    }
}

/* ---------------------------------------------------------- voxel keys -- */

/* Transformed point q = T p by the fixed fma chain, and its voxel coordinate.
 * Returns 1 if the coordinate is valid. */
static int voxel_coord(const double *T, const float *p, double inv_r, double q[3], int64_t k[3])
{
    const double px = (double)p[0], py = (double)p[1], pz = (double)p[2];
    int ok = 1;
    for (int i = 0; i < 3; ++i) {
        q[i] = fma(T[4 * i + 0], px, fma(T[4 * i + 1], py, fma(T[4 * i + 2], pz, T[4 * i + 3])));
        double f = floor(q[i] * inv_r);
        if (!(f >= KEY_MIN && f <= KEY_MAX)) { ok = 0; k[i] = 0; }
        else k[i] = (int64_t)f;
    }
    return ok;
}

/* Per-point voxel coordinates of a cloud under pose T (identity when T is NULL). */
void oracle_voxel_coords(const float *pts, int64_t n, const double *T, double r,
                         int64_t *coords, int32_t *valid)
{
    static const double I[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    const double inv_r = 1.0 / r;
    double q[3];
    for (int64_t i = 0; i < n; ++i)
        valid[i] = voxel_coord(T ? T : I, pts + 3 * i, inv_r, q, coords + 3 * i);
}

static int key_cmp(const int64_t *a, const int64_t *b)
{
    for (int i = 0; i < 3; ++i) {
        if (a[i] < b[i]) return -1;
        if (a[i] > b[i]) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------ voxelmap -- */

typedef struct { int64_t k[3]; int64_t idx; } keyed_t;

static int keyed_cmp(const void *pa, const void *pb)
{
    const keyed_t *a = (const keyed_t *)pa, *b = (const keyed_t *)pb;
    int c = key_cmp(a->k, b->k);
    if (c) return c;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

/* Voxelmap of a cloud in its own frame at resolution r (Sec. III-A).
 * Output voxels are sorted by (kx, ky, kz); all output arrays have room for n
 * voxels.  Sums run over each voxel's points in increasing point index.
 * Returns the number of voxels. */
int64_t oracle_voxelmap_build(const float *pts, const float *covs, int64_t n, double r,
                              int64_t *keys, int64_t *counts, double *mu, double *cov)
{
    keyed_t *kv = (keyed_t *)malloc(sizeof(keyed_t) * (size_t)(n > 0 ? n : 1));
    int64_t m = 0;
    static const double I[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    const double inv_r = 1.0 / r;
    double q[3];
    for (int64_t i = 0; i < n; ++i) {
        if (voxel_coord(I, pts + 3 * i, inv_r, q, kv[m].k)) { kv[m].idx = i; ++m; }
    }
    qsort(kv, (size_t)m, sizeof(keyed_t), keyed_cmp);
    int64_t nv = 0;
    for (int64_t s = 0; s < m;) {
        int64_t e = s;
        double sm[3] = {0, 0, 0}, sc[6] = {0, 0, 0, 0, 0, 0};
        while (e < m && key_cmp(kv[e].k, kv[s].k) == 0) {
            const int64_t i = kv[e].idx;
            for (int d = 0; d < 3; ++d) sm[d] = sm[d] + (double)pts[3 * i + d];
            for (int d = 0; d < 6; ++d) sc[d] = sc[d] + (double)covs[6 * i + d];
            ++e;
        }
        const double c = (double)(e - s);
        for (int d = 0; d < 3; ++d) { keys[3 * nv + d] = kv[s].k[d]; mu[3 * nv + d] = sm[d] / c; }
        for (int d = 0; d < 6; ++d) cov[6 * nv + d] = sc[d] / c;
        counts[nv] = e - s;
        ++nv;
        s = e;
    }
    free(kv);
    return nv;
}

/* The same voxelmap by brute force: a linear list of keys in first-seen order,
 * each point searched against every key seen so far. */
int64_t oracle_voxelmap_build_bruteforce(const float *pts, const float *covs, int64_t n, double r,
                                         int64_t *keys, int64_t *counts, double *mu, double *cov)
{
    static const double I[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    const double inv_r = 1.0 / r;
    double q[3];
    int64_t k[3], nv = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!voxel_coord(I, pts + 3 * i, inv_r, q, k)) continue;
        int64_t v = 0;
        while (v < nv && key_cmp(keys + 3 * v, k) != 0) ++v;
        if (v == nv) {
            memcpy(keys + 3 * v, k, sizeof(k));
            counts[v] = 0;
            for (int d = 0; d < 3; ++d) mu[3 * v + d] = 0.0;
            for (int d = 0; d < 6; ++d) cov[6 * v + d] = 0.0;
            ++nv;
        }
        counts[v] += 1;
        for (int d = 0; d < 3; ++d) mu[3 * v + d] = mu[3 * v + d] + (double)pts[3 * i + d];
        for (int d = 0; d < 6; ++d) cov[6 * v + d] = cov[6 * v + d] + (double)covs[6 * i + d];
    }
    for (int64_t v = 0; v < nv; ++v) {
        for (int d = 0; d < 3; ++d) mu[3 * v + d] = mu[3 * v + d] / (double)counts[v];
        for (int d = 0; d < 6; ++d) cov[6 * v + d] = cov[6 * v + d] / (double)counts[v];
    }
    return nv;
}

/* Index of voxel k in a sorted key list, or -1 (binary search). */
int64_t oracle_lookup(const int64_t *keys, int64_t nv, const int64_t *k)
{
    int64_t lo = 0, hi = nv - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int c = key_cmp(keys + 3 * mid, k);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Index of voxel k in any key list, or -1 (linear search). */
int64_t oracle_lookup_bruteforce(const int64_t *keys, int64_t nv, const int64_t *k)
{
    for (int64_t v = 0; v < nv; ++v)
        if (key_cmp(keys + 3 * v, k) == 0) return v;
    return -1;
}

/* Correspondence of every source point: the target voxel containing T_BA p
 * (Sec. III-A: look-up in the target voxelmap, no neighbour voxels), or -1.
 * keys_out (n x 3, nullable) receives the voxel coordinates. */
void oracle_correspondences(const int64_t *keys, int64_t nv, double r,
                            const float *src, int64_t n, const double *TBA,
                            int64_t *corr, int64_t *keys_out)
{
    const double inv_r = 1.0 / r;
    double q[3];
    int64_t k[3];
    for (int64_t i = 0; i < n; ++i) {
        int ok = voxel_coord(TBA, src + 3 * i, inv_r, q, k);
        corr[i] = ok ? oracle_lookup(keys, nv, k) : -1;
        if (keys_out) { for (int d = 0; d < 3; ++d) keys_out[3 * i + d] = ok ? k[d] : INT64_MIN; }
    }
}

/* Overlap (Eq. 7-8): number of source points whose transformed point falls in
 * a voxel of the target map.  The fraction is this count divided by n. */
int64_t oracle_overlap_count(const int64_t *keys, int64_t nv, double r,
                             const float *src, int64_t n, const double *TBA)
{
    const double inv_r = 1.0 / r;
    double q[3];
    int64_t k[3], count = 0;
    for (int64_t i = 0; i < n; ++i)
        if (voxel_coord(TBA, src + 3 * i, inv_r, q, k) && oracle_lookup(keys, nv, k) >= 0) ++count;
    return count;
}

/* -------------------------------------------------- per-point GICP term -- */

static void cov_full(const float *c, double M[3][3])
{
    M[0][0] = c[0]; M[0][1] = c[1]; M[0][2] = c[2];
    M[1][0] = c[1]; M[1][1] = c[3]; M[1][2] = c[4];
    M[2][0] = c[2]; M[2][1] = c[4]; M[2][2] = c[5];
}

static void cov_full_d(const double *c, double M[3][3])
{
    M[0][0] = c[0]; M[0][1] = c[1]; M[0][2] = c[2];
    M[1][0] = c[1]; M[1][1] = c[3]; M[1][2] = c[4];
    M[2][0] = c[2]; M[2][1] = c[4]; M[2][2] = c[5];
}

/* Inverse of a symmetric positive definite 3x3 by Cholesky factorisation and
 * forward/back substitution against the identity.  Returns 0 if M is not PD. */
static int spd_inverse(double M[3][3], double W[3][3])
{
    double L[3][3] = {{0}};
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = M[i][j];
            for (int k = 0; k < j; ++k) s = s - L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 0.0)) return 0;
                L[i][i] = sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    }
    for (int c = 0; c < 3; ++c) {
        double y[3], x[3];
        for (int i = 0; i < 3; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s = s - L[i][k] * y[k];
            y[i] = s / L[i][i];
        }
        for (int i = 2; i >= 0; --i) {
            double s = y[i];
            for (int k = i + 1; k < 3; ++k) s = s - L[k][i] * x[k];
            x[i] = s / L[i][i];
        }
        for (int i = 0; i < 3; ++i) W[i][c] = x[i];
    }
    return 1;
}

/* One correspondence: residual e = mu_B - q (Eq. 2), Omega = (C_B + R C_A R^T)^-1
 * and the 3x12 Jacobian J = [de/dxi_B | de/dxi_A] = [-[q]x, I | R[p]x, -R]. */
static int point_term(const double *T, const float *p, const float *ca,
                      const double *mu_b, const double *cov_b, const double q[3],
                      double e[3], double Om[3][3], double J[3][12])
{
    double R[3][3], CA[3][3], CB[3][3], RC[3][3], M[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[i][j] = T[4 * i + j];
    cov_full(ca, CA);
    cov_full_d(cov_b, CB);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s = s + R[i][k] * CA[k][j];
            RC[i][j] = s;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s = s + RC[i][k] * R[j][k];
            M[i][j] = CB[i][j] + s;
        }
    if (!spd_inverse(M, Om)) return 0;
    for (int i = 0; i < 3; ++i) e[i] = mu_b[i] - q[i];
    const double px = p[0], py = p[1], pz = p[2];
    const double P[3][3] = {{0, -pz, py}, {pz, 0, -px}, {-py, px, 0}};         /* [p]x */
    const double Q[3][3] = {{0, -q[2], q[1]}, {q[2], 0, -q[0]}, {-q[1], q[0], 0}}; /* [q]x */
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double rp = 0.0;
            for (int k = 0; k < 3; ++k) rp = rp + R[i][k] * P[k][j];
            J[i][j] = -Q[i][j];
            J[i][3 + j] = (i == j) ? 1.0 : 0.0;
            J[i][6 + j] = rp;
            J[i][9 + j] = -R[i][j];
        }
    }
    return 1;
}

/* Voxel offsets searched around a point's own voxel k: DIRECT1 = {0};
 * DIRECT7 = k and its six face neighbours; DIRECT27 = the 3x3x3 block.  Listed
 * as: (0,0,0), then -x, +x, -y, +y, -z, +z, then the remaining twenty with
 * x outermost, each coordinate running -1, 0, 1. */
static int neighbour_offsets(int nb, int off[27][3])
{
    static const int face[7][3] = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    int m = 0;
    for (int i = 0; i < 7 && i < nb; ++i, ++m)
        for (int a = 0; a < 3; ++a) off[m][a] = face[i][a];
    if (nb == 27)
        for (int x = -1; x <= 1; ++x)
            for (int y = -1; y <= 1; ++y)
                for (int z = -1; z <= 1; ++z) {
                    if (abs(x) + abs(y) + abs(z) <= 1) continue;
                    off[m][0] = x;
                    off[m][1] = y;
                    off[m][2] = z;
                    ++m;
                }
    return m;
}

/* Linearisation of one factor (Eq. 3-6): cost = sum e^T Omega e,
 * H = sum J^T Omega J (12x12, full), b = sum J^T Omega e, over every
 * correspondence (source point, target voxel).  nb = 1: the voxel containing
 * the transformed point (Sec. III-A); nb = 7 or 27: also its face neighbours
 * or its whole 3x3x3 block (the DIRECT7 / DIRECT27 association of the earlier
 * VGICP paper), each neighbour a correspondence of its own with e = mu_v - q.
 * counts != NULL weights each correspondence by its voxel's point count.
 * S* receive the sums of the absolute per-correspondence contributions (the
 * scale used by the error metric); inliers counts correspondences.  corr (n,
 * nullable) receives each point's containing-voxel index or -1. */
void oracle_linearize_ex(const int64_t *keys, const double *mu, const double *cov, const int64_t *counts,
                         int64_t nv, double r, int nb, const float *src, const float *src_cov, int64_t n,
                         const double *TBA, double *H, double *b, double *cost, int64_t *inliers, double *SH,
                         double *Sb, double *Scost, int64_t *corr)
{
    const double inv_r = 1.0 / r;
    int off[27][3];
    const int no = neighbour_offsets(nb, off);
    memset(H, 0, sizeof(double) * 144);
    memset(b, 0, sizeof(double) * 12);
    if (SH) memset(SH, 0, sizeof(double) * 144);
    if (Sb) memset(Sb, 0, sizeof(double) * 12);
    double c = 0.0, sc = 0.0;
    int64_t in = 0;
    for (int64_t i = 0; i < n; ++i) {
        double q[3], e[3], Om[3][3], J[3][12];
        int64_t k[3];
        const int valid = voxel_coord(TBA, src + 3 * i, inv_r, q, k);
        if (corr) corr[i] = valid ? oracle_lookup(keys, nv, k) : -1;
        if (!valid) continue;
        for (int o = 0; o < no; ++o) {
            int64_t kk[3];
            int inside = 1;
            for (int a = 0; a < 3; ++a) {
                kk[a] = k[a] + off[o][a];
                inside = inside && kk[a] >= -1048576 && kk[a] <= 1048575;
            }
            const int64_t v = inside ? oracle_lookup(keys, nv, kk) : -1;
            if (v < 0) continue;
            if (!point_term(TBA, src + 3 * i, src_cov + 6 * i, mu + 3 * v, cov + 6 * v, q, e, Om, J)) continue;
            if (counts) {
                const double w = (double)counts[v];
                for (int a = 0; a < 3; ++a)
                    for (int m = 0; m < 3; ++m) Om[a][m] = Om[a][m] * w;
            }
            double OJ[3][12], Oe[3];
            for (int a = 0; a < 3; ++a) {
                for (int j = 0; j < 12; ++j) {
                    double s = 0.0;
                    for (int m = 0; m < 3; ++m) s = s + Om[a][m] * J[m][j];
                    OJ[a][j] = s;
                }
                double s = 0.0;
                for (int m = 0; m < 3; ++m) s = s + Om[a][m] * e[m];
                Oe[a] = s;
            }
            double ck = 0.0;
            for (int a = 0; a < 3; ++a) ck = ck + e[a] * Oe[a];
            c = c + ck;
            sc = sc + fabs(ck);
            for (int a = 0; a < 12; ++a) {
                for (int j = a; j < 12; ++j) {   /* upper triangle; H is symmetric by definition */
                    double s = 0.0;
                    for (int m = 0; m < 3; ++m) s = s + J[m][a] * OJ[m][j];
                    H[12 * a + j] = H[12 * a + j] + s;
                    if (SH) SH[12 * a + j] = SH[12 * a + j] + fabs(s);
                }
                double s = 0.0;
                for (int m = 0; m < 3; ++m) s = s + J[m][a] * Oe[m];
                b[a] = b[a] + s;
                if (Sb) Sb[a] = Sb[a] + fabs(s);
            }
            ++in;
        }
    }
    for (int a = 0; a < 12; ++a)
        for (int j = 0; j < a; ++j) {
            H[12 * a + j] = H[12 * j + a];
            if (SH) SH[12 * a + j] = SH[12 * j + a];
        }
    *cost = c;
    if (Scost) *Scost = sc;
    if (inliers) *inliers = in;
}

/* The single-voxel, unweighted linearisation (Sec. III-A association). */
void oracle_linearize(const int64_t *keys, const double *mu, const double *cov, int64_t nv, double r,
                      const float *src, const float *src_cov, int64_t n, const double *TBA,
                      double *H, double *b, double *cost, int64_t *inliers,
                      double *SH, double *Sb, double *Scost, int64_t *corr)
{
    oracle_linearize_ex(keys, mu, cov, NULL, nv, r, 1, src, src_cov, n, TBA, H, b, cost, inliers, SH, Sb, Scost,
                        corr);
}

/* Per-point residuals and Jacobians under a frozen correspondence list corr
 * (voxel index per point, -1 = none) and a frozen pose T_lin for Omega: for
 * finite-difference checks.  e (n x 3), J (n x 36, nullable) are zero where
 * corr < 0.  q is formed by the same fma chain as the voxel coordinate. */
void oracle_residuals(const double *mu, const double *cov, const float *src, const float *src_cov,
                      int64_t n, const double *TBA, const int64_t *corr, double *e_out, double *J_out,
                      double *Om_out)
{
    for (int64_t i = 0; i < n; ++i) {
        double q[3], e[3], Om[3][3], J[3][12];
        memset(e_out + 3 * i, 0, sizeof(double) * 3);
        if (J_out) memset(J_out + 36 * i, 0, sizeof(double) * 36);
        if (Om_out) memset(Om_out + 9 * i, 0, sizeof(double) * 9);
        if (corr[i] < 0) continue;
        const float *p = src + 3 * i;
        for (int a = 0; a < 3; ++a)
            q[a] = fma(TBA[4 * a + 0], (double)p[0], fma(TBA[4 * a + 1], (double)p[1],
                   fma(TBA[4 * a + 2], (double)p[2], TBA[4 * a + 3])));
        if (!point_term(TBA, p, src_cov + 6 * i, mu + 3 * corr[i], cov + 6 * corr[i], q, e, Om, J)) continue;
        for (int a = 0; a < 3; ++a) e_out[3 * i + a] = e[a];
        if (J_out) for (int a = 0; a < 3; ++a) for (int j = 0; j < 12; ++j) J_out[36 * i + 12 * a + j] = J[a][j];
        if (Om_out) for (int a = 0; a < 3; ++a) for (int j = 0; j < 3; ++j) Om_out[9 * i + 3 * a + j] = Om[a][j];
    }
}

/* --------------------------------------------- k-nearest-neighbour covariances -- */

/* Squared distance between two float points, promoted to double; sum order
 * ((dx*dx + dy*dy) + dz*dz), each operation separately rounded. */
static double dist2(const float *a, const float *b)
{
    const double dx = (double)a[0] - (double)b[0];
    const double dy = (double)a[1] - (double)b[1];
    const double dz = (double)a[2] - (double)b[2];
    return (dx * dx + dy * dy) + dz * dz;
}

/* (d, j) < (d', j'): smaller distance first, ties to the lower index. */
static int nb_less(double d, int64_t j, double d2, int64_t j2)
{
    return (d < d2) || (d == d2 && j < j2);
}

static void nb_insert(double *bd, int64_t *bj, int *cnt, int k, double d, int64_t j)
{
    if (*cnt == k && !nb_less(d, j, bd[k - 1], bj[k - 1])) return;
    int pos = (*cnt < k) ? (*cnt)++ : k - 1;
    while (pos > 0 && nb_less(d, j, bd[pos - 1], bj[pos - 1])) {
        bd[pos] = bd[pos - 1];
        bj[pos] = bj[pos - 1];
        --pos;
    }
    bd[pos] = d;
    bj[pos] = j;
}

/* k nearest neighbours of every point (the point itself included) by checking
 * every pair.  nbr is n x k, nearest first. */
void oracle_knn_bruteforce(const float *pts, int64_t n, int k, int64_t *nbr)
{
    double *bd = (double *)malloc(sizeof(double) * (size_t)k);
    for (int64_t i = 0; i < n; ++i) {
        int cnt = 0;
        for (int64_t j = 0; j < n; ++j) nb_insert(bd, nbr + (size_t)k * i, &cnt, k, dist2(pts + 3 * i, pts + 3 * j), j);
        for (int c = cnt; c < k; ++c) nbr[(size_t)k * i + c] = -1;
    }
    free(bd);
}

typedef struct { int64_t c[3]; int64_t idx; } cell_t;

static int cell_cmp(const void *pa, const void *pb)
{
    const cell_t *a = (const cell_t *)pa, *b = (const cell_t *)pb;
    int c = key_cmp(a->c, b->c);
    if (c) return c;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

static int64_t cell_first(const cell_t *cs, int64_t m, const int64_t *c)
{
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (key_cmp(cs[mid].c, c) < 0) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* The same k nearest neighbours with a uniform grid of cell size h: cubes of
 * cells around the query grow shell by shell until every point not yet seen is
 * provably farther than the current k-th neighbour (after 16 shells the query
 * scans every point instead).  Points with non-finite coordinates get no
 * neighbours (-1). */
void oracle_knn_grid(const float *pts, int64_t n, int k, double h, int64_t *nbr)
{
    cell_t *cs = (cell_t *)malloc(sizeof(cell_t) * (size_t)(n > 0 ? n : 1));
    int64_t m = 0, lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {INT64_MIN, INT64_MIN, INT64_MIN};
    for (int64_t i = 0; i < n; ++i) {
        int ok = 1;
        for (int d = 0; d < 3; ++d) ok &= isfinite(pts[3 * i + d]);
        if (!ok) continue;
        for (int d = 0; d < 3; ++d) {
            cs[m].c[d] = (int64_t)floor((double)pts[3 * i + d] / h);
            if (cs[m].c[d] < lo[d]) lo[d] = cs[m].c[d];
            if (cs[m].c[d] > hi[d]) hi[d] = cs[m].c[d];
        }
        cs[m].idx = i;
        ++m;
    }
    qsort(cs, (size_t)m, sizeof(cell_t), cell_cmp);
    int64_t span = 0;
    for (int d = 0; d < 3; ++d) if (m && hi[d] - lo[d] > span) span = hi[d] - lo[d];
    double *bd = (double *)malloc(sizeof(double) * (size_t)k);
    for (int64_t i = 0; i < n; ++i) {
        int64_t *out = nbr + (size_t)k * i;
        int cnt = 0, ok = 1;
        for (int d = 0; d < 3; ++d) ok &= isfinite(pts[3 * i + d]);
        if (ok) {
            int64_t c0[3];
            for (int d = 0; d < 3; ++d) c0[d] = (int64_t)floor((double)pts[3 * i + d] / h);
            for (int64_t s = 0;; ++s) {
                if (s > 16) {
                    /* sparse neighbourhood: scan every point instead */
                    cnt = 0;
                    for (int64_t j = 0; j < n; ++j) {
                        int fin = 1;
                        for (int d = 0; d < 3; ++d) fin &= isfinite(pts[3 * j + d]);
                        if (fin) nb_insert(bd, out, &cnt, k, dist2(pts + 3 * i, pts + 3 * j), j);
                    }
                    break;
                }
                /* visit the cells at Chebyshev distance exactly s from c0 (the shell's surface) */
                for (int64_t dx = -s; dx <= s; ++dx)
                    for (int64_t dy = -s; dy <= s; ++dy) {
                        const int edge = (llabs(dx) == s || llabs(dy) == s);
                        for (int64_t dz = -s; dz <= s; dz += (edge || s == 0) ? 1 : 2 * s) {
                            int64_t c[3] = {c0[0] + dx, c0[1] + dy, c0[2] + dz};
                            for (int64_t t = cell_first(cs, m, c); t < m && key_cmp(cs[t].c, c) == 0; ++t)
                                nb_insert(bd, out, &cnt, k, dist2(pts + 3 * i, pts + 3 * cs[t].idx), cs[t].idx);
                        }
                    }
                /* everything unseen is at distance >= s*h from the query */
                const double reach = (double)s * h;
                if (cnt == k && bd[k - 1] < reach * reach * (1.0 - 1e-9)) break;
                if (s > span + 1) break;
            }
        }
        for (int c = cnt; c < k; ++c) out[c] = -1;
    }
    free(bd);
    free(cs);
}

/* Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (Golub and
 * Van Loan, Matrix Computations, Sec. 8.5): A = V diag(w) V^T.  Sweeps until
 * the off-diagonal Frobenius norm is below 1e-15 of the matrix norm. */
void oracle_jacobi_eig3(const double *Ain, double *w, double *V)
{
    double A[3][3], U[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    double nrm = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { A[i][j] = Ain[3 * i + j]; nrm += A[i][j] * A[i][j]; }
    nrm = sqrt(nrm);
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = sqrt(2.0 * (A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2]));
        if (off <= 1e-15 * nrm || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                /* rotation (c, s) that zeroes A[p][q] (symmetric Schur decomposition) */
                double tau = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < 3; ++k) {       /* A <- A J */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {       /* A <- J^T A */
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {       /* V <- V J */
                    double ukp = U[k][p], ukq = U[k][q];
                    U[k][p] = c * ukp - s * ukq;
                    U[k][q] = s * ukp + c * ukq;
                }
            }
    }
    for (int i = 0; i < 3; ++i) {
        w[i] = A[i][i];
        for (int j = 0; j < 3; ++j) V[3 * i + j] = U[i][j];
    }
}

/* Per-point covariance from its k nearest neighbours (Sec. III: estimated from
 * k neighbouring points), regularised to eigenvalues (1, 1, eps): the sample
 * covariance about the neighbour mean is diagonalised, eigenvalues sorted in
 * decreasing order (stable in column index), and C = U diag(1, 1, eps) U^T, so
 * the direction of least spread (the surface normal) receives eps.  Points
 * without k neighbours get the identity.  covs is n x 6 float32. */
void oracle_covariances_from_neighbors(const float *pts, int64_t n, int k, const int64_t *nbr,
                                       double eps, float *covs)
{
    for (int64_t i = 0; i < n; ++i) {
        const int64_t *nb = nbr + (size_t)k * i;
        int full = 1;
        for (int j = 0; j < k; ++j) full &= nb[j] >= 0;
        float *out = covs + 6 * i;
        if (!full) {
            out[0] = 1; out[1] = 0; out[2] = 0; out[3] = 1; out[4] = 0; out[5] = 1;
            continue;
        }
        double m[3] = {0, 0, 0};
        for (int j = 0; j < k; ++j)
            for (int d = 0; d < 3; ++d) m[d] = m[d] + (double)pts[3 * nb[j] + d];
        for (int d = 0; d < 3; ++d) m[d] = m[d] / (double)k;
        double S[9] = {0};
        for (int j = 0; j < k; ++j) {
            double x[3];
            for (int d = 0; d < 3; ++d) x[d] = (double)pts[3 * nb[j] + d] - m[d];
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) S[3 * a + c] = S[3 * a + c] + x[a] * x[c];
        }
        for (int a = 0; a < 9; ++a) S[a] = S[a] / (double)k;
        double w[3], V[9];
        oracle_jacobi_eig3(S, w, V);
        int ord[3] = {0, 1, 2};
        for (int a = 1; a < 3; ++a) {             /* stable insertion sort, descending */
            int t = ord[a], p = a;
            while (p > 0 && w[ord[p - 1]] < w[t]) { ord[p] = ord[p - 1]; --p; }
            ord[p] = t;
        }
        const double lam[3] = {1.0, 1.0, eps};
        double C[3][3];
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int j = 0; j < 3; ++j) s = s + V[3 * a + ord[j]] * lam[j] * V[3 * c + ord[j]];
                C[a][c] = s;
            }
        out[0] = (float)C[0][0]; out[1] = (float)C[0][1]; out[2] = (float)C[0][2];
        out[3] = (float)C[1][1]; out[4] = (float)C[1][2]; out[5] = (float)C[2][2];
    }
}
