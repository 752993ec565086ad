// Per-point covariance from the k nearest neighbours (Sec. III: estimated from
// k neighbouring points once per input cloud), regularised to eigenvalues
// (1, 1, eps) so the surface normal direction receives eps.
//
// Neighbour search: every query scans every point of its cloud in shared-memory
// tiles.  Squared distances are formed in float64 as ((dx*dx + dy*dy) + dz*dz),
// each operation separately rounded, so the neighbour set (ties to the lower
// index) is exactly that of the definition.  The 3x3 eigen-decomposition is
// cyclic Jacobi in float64.
#include "kernels.cuh"

namespace vg {

namespace {

constexpr int kTile = 256;
constexpr int kMaxK = 32;

__device__ __forceinline__ bool nb_less(double d, int64_t j, double d2, int64_t j2)
{
    return (d < d2) || (d == d2 && j < j2);
}

__device__ __forceinline__ bool finite3(float x, float y, float z)
{
    return isfinite(x) && isfinite(y) && isfinite(z);
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

__global__ void __launch_bounds__(kTile) k_knn_cov(const float *__restrict__ pts, int64_t n, int k, double eps,
                                                   float *__restrict__ covs)
{
    __shared__ float sx[kTile], sy[kTile], sz[kTile];
    const int64_t i = blockIdx.x * (int64_t)kTile + threadIdx.x;
    const bool active = i < n;
    float qx = 0.f, qy = 0.f, qz = 0.f;
    if (active) { qx = pts[3 * i]; qy = pts[3 * i + 1]; qz = pts[3 * i + 2]; }
    const bool query = active && finite3(qx, qy, qz);
    double bd[kMaxK];
    int64_t bj[kMaxK];
    int cnt = 0;
    for (int64_t t0 = 0; t0 < n; t0 += kTile) {
        __syncthreads();
        const int64_t j = t0 + threadIdx.x;
        if (j < n) { sx[threadIdx.x] = pts[3 * j]; sy[threadIdx.x] = pts[3 * j + 1]; sz[threadIdx.x] = pts[3 * j + 2]; }
        __syncthreads();
        if (!query) continue;
        const int m = (n - t0 < kTile) ? (int)(n - t0) : kTile;
        for (int c = 0; c < m; ++c) {
            const float x = sx[c], y = sy[c], z = sz[c];
            if (!finite3(x, y, z)) continue;
            const double dx = __dsub_rn((double)qx, (double)x);
            const double dy = __dsub_rn((double)qy, (double)y);
            const double dz = __dsub_rn((double)qz, (double)z);
            const double d = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            const int64_t jj = t0 + c;
            if (cnt == k && !nb_less(d, jj, bd[k - 1], bj[k - 1])) continue;
            int pos = (cnt < k) ? cnt++ : k - 1;
            while (pos > 0 && nb_less(d, jj, bd[pos - 1], bj[pos - 1])) {
                bd[pos] = bd[pos - 1];
                bj[pos] = bj[pos - 1];
                --pos;
            }
            bd[pos] = d;
            bj[pos] = jj;
        }
    }
    if (!active) return;
    float *out = covs + 6 * i;
    if (cnt < k) {
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

void launch_knn_covariances(const float *points, int64_t n, int k, double eps, float *covs, cudaStream_t st)
{
    if (n <= 0) return;
    k_knn_cov<<<(unsigned)((n + kTile - 1) / kTile), kTile, 0, st>>>(points, n, k, eps, covs);
}

}  // namespace vg
