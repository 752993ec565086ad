// Gauss-Newton / Levenberg-Marquardt over the VGICP factors (Sec. III-D: the
// global optimisation linearises every factor on the GPU, collects the linear
// system and solves it on the host).
//
//   * vgicp_solve_step: the damped normal equations (H + lambda diag(H)) d = -b
//     of a factor set, assembled from the factors' 12x12 blocks, with one pose
//     held fixed (the gauge), solved by a sparse Cholesky factorisation: poses
//     are ordered by reverse Cuthill-McKee on the pose graph, so the factor
//     stays inside the band of the matrix's envelope (skyline storage).
//   * vgicp_se3_retract: T <- T Exp(d) per pose (right perturbation, d = (omega, v)).
//   * vgicp_optimize: the Levenberg-Marquardt loop; each iteration linearises
//     through a plan (one CUDA graph), solves on the host, evaluates the cost of
//     the trial poses with the cost-only pass and accepts or rejects the step.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <vector>

#include "envelope_cholesky.h"
#include "vgicp.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0) { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }

// Reverse Cuthill-McKee order of the graph's nodes (every component).
std::vector<int> rcm_order(const std::vector<std::vector<int>> &adj)
{
    const int n = (int)adj.size();
    std::vector<int> order, deg(n);
    std::vector<char> seen(n, 0);
    for (int i = 0; i < n; ++i) deg[i] = (int)adj[i].size();
    order.reserve(n);
    for (;;) {
        int start = -1;
        for (int i = 0; i < n; ++i)
            if (!seen[i] && (start < 0 || deg[i] < deg[start])) start = i;
        if (start < 0) break;
        // move the start to a pseudo-peripheral node: the last node of a BFS, twice
        for (int pass = 0; pass < 2; ++pass) {
            std::vector<char> vis(n, 0);
            std::deque<int> q{start};
            vis[start] = 1;
            int last = start;
            while (!q.empty()) {
                const int u = q.front();
                q.pop_front();
                last = u;
                for (int v : adj[u])
                    if (!vis[v] && !seen[v]) {
                        vis[v] = 1;
                        q.push_back(v);
                    }
            }
            start = last;
        }
        std::deque<int> q{start};
        seen[start] = 1;
        while (!q.empty()) {
            const int u = q.front();
            q.pop_front();
            order.push_back(u);
            std::vector<int> nb;
            for (int v : adj[u])
                if (!seen[v]) {
                    seen[v] = 1;
                    nb.push_back(v);
                }
            std::sort(nb.begin(), nb.end(), [&](int a, int b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; });
            for (int v : nb) q.push_back(v);
        }
    }
    std::reverse(order.begin(), order.end());
    return order;
}

// Symmetric matrix in skyline (envelope) storage by rows: row r holds columns
// first[r] .. r contiguously.
struct Skyline {
    std::vector<int64_t> first, off;
    std::vector<double> a;
    double &at(int64_t r, int64_t c) { return a[off[r] + (c - first[r])]; }
};

// The global system's product H x from the factor blocks (x, y: 6 per pose).
void global_matvec(const int32_t *pairs, const double *H, int64_t n_f, const double *x, double *y, int64_t n_poses)
{
    std::fill(y, y + 6 * n_poses, 0.0);
    for (int64_t f = 0; f < n_f; ++f) {
        const int32_t pose[2] = {pairs[2 * f], pairs[2 * f + 1]};
        const double *Hf = H + 144 * f;
        for (int bi = 0; bi < 2; ++bi)
            for (int r = 0; r < 6; ++r) {
                double s = 0.0;
                for (int bj = 0; bj < 2; ++bj)
                    for (int c = 0; c < 6; ++c) s += Hf[12 * (6 * bi + r) + 6 * bj + c] * x[6 * pose[bj] + c];
                y[6 * pose[bi] + r] += s;
            }
    }
}

void so3_exp(const double w[3], double R[9])
{
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2], th = std::sqrt(th2);
    double A, B;   // sin(th) / th, (1 - cos(th)) / th^2
    if (th < 1e-4) {
        A = 1.0 - th2 / 6.0;
        B = 0.5 - th2 / 24.0;
    } else {
        A = std::sin(th) / th;
        B = (1.0 - std::cos(th)) / th2;
    }
    const double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double KK = 0.0;
            for (int k = 0; k < 3; ++k) KK += K[3 * i + k] * K[3 * k + j];
            R[3 * i + j] = (i == j ? 1.0 : 0.0) + A * K[3 * i + j] + B * KK;
        }
}

// Exp of a twist (omega, v): rotation and translation V v with
// V = I + B [w]x + C [w]x^2, B = (1 - cos) / th^2, C = (th - sin) / th^3.
void se3_exp(const double xi[6], double T[12])
{
    double R[9];
    so3_exp(xi, R);
    const double *w = xi, *v = xi + 3;
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2], th = std::sqrt(th2);
    double B, C;
    if (th < 1e-4) {
        B = 0.5 - th2 / 24.0;
        C = 1.0 / 6.0 - th2 / 120.0;
    } else {
        B = (1.0 - std::cos(th)) / th2;
        C = (th - std::sin(th)) / (th2 * th);
    }
    const double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    for (int i = 0; i < 3; ++i) {
        double t = v[i];
        for (int j = 0; j < 3; ++j) {
            double KK = 0.0;
            for (int k = 0; k < 3; ++k) KK += K[3 * i + k] * K[3 * k + j];
            t += (B * K[3 * i + j] + C * KK) * v[j];
        }
        for (int j = 0; j < 3; ++j) T[4 * i + j] = R[3 * i + j];
        T[4 * i + 3] = t;
    }
}

// ---------------------------------------------------------- SE(3) helpers --

void compose34(const double A[12], const double B[12], double C[12])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = j == 3 ? A[4 * i + 3] : 0.0;
            for (int k = 0; k < 3; ++k) s += A[4 * i + k] * B[4 * k + j];
            C[4 * i + j] = s;
        }
}

void invert34(const double T[12], double Ti[12])
{
    for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) {
            Ti[4 * i + k] = T[4 * k + i];
            s -= T[4 * k + i] * T[4 * k + 3];
        }
        Ti[4 * i + 3] = s;
    }
}

void skew(const double a[3], double K[9])
{
    K[0] = 0.0;   K[1] = -a[2]; K[2] = a[1];
    K[3] = a[2];  K[4] = 0.0;   K[5] = -a[0];
    K[6] = -a[1]; K[7] = a[0];  K[8] = 0.0;
}

// Log of a rotation (axis-angle), robust at 0 and at pi.
void so3_log(const double R[9], double w[3])
{
    const double c = std::max(-1.0, std::min(1.0, 0.5 * (R[0] + R[4] + R[8] - 1.0)));
    const double th = std::acos(c);
    const double v[3] = {R[7] - R[5], R[2] - R[6], R[3] - R[1]};
    if (th < 1e-5) {
        for (int a = 0; a < 3; ++a) w[a] = 0.5 * (1.0 + th * th / 6.0) * v[a];
    } else if (M_PI - th < 1e-5) {
        int k = 0;
        for (int a = 1; a < 3; ++a)
            if (R[4 * a] > R[4 * k]) k = a;
        const double d = std::sqrt(2.0 * (1.0 + R[4 * k]));
        for (int a = 0; a < 3; ++a) w[a] = th * (R[3 * a + k] + (a == k ? 1.0 : 0.0)) / d;
    } else {
        const double f = th / (2.0 * std::sin(th));
        for (int a = 0; a < 3; ++a) w[a] = f * v[a];
    }
}

// Log of a rigid transform as a twist (omega, v): v = V(omega)^-1 t.
void se3_log(const double T[12], double xi[6])
{
    const double R[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
    so3_log(R, xi);
    const double th2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2], th = std::sqrt(th2);
    double c;   // coefficient of [w]x^2 in V^-1
    if (th < 1e-4) c = 1.0 / 12.0 + th2 / 720.0;
    else c = (1.0 - th * std::sin(th) / (2.0 * (1.0 - std::cos(th)))) / th2;
    double K[9];
    skew(xi, K);
    const double t[3] = {T[3], T[7], T[11]};
    for (int i = 0; i < 3; ++i) {
        double s = t[i];
        for (int j = 0; j < 3; ++j) {
            double KK = 0.0;
            for (int k = 0; k < 3; ++k) KK += K[3 * i + k] * K[3 * k + j];
            s += (-0.5 * K[3 * i + j] + c * KK) * t[j];
        }
        xi[3 + i] = s;
    }
}

// Adjoint of T on twists (omega, v): [[R, 0], [[t]x R, R]] (6x6 row-major).
void adjoint(const double T[12], double Ad[36])
{
    double tx[9];
    const double t[3] = {T[3], T[7], T[11]};
    skew(t, tx);
    std::fill(Ad, Ad + 36, 0.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const double r = T[4 * i + j];
            Ad[6 * i + j] = r;
            Ad[6 * (3 + i) + 3 + j] = r;
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += tx[3 * i + k] * T[4 * k + j];
            Ad[6 * (3 + i) + j] = s;
        }
}

// Inverse right Jacobian of SE(3) to second order: I + ad/2 + ad^2/12 with
// ad(omega, v) = [[ [w]x, 0 ], [ [v]x, [w]x ]].
void jr_inverse(const double xi[6], double J[36])
{
    double a[36] = {0}, W[9], V[9];
    skew(xi, W);
    skew(xi + 3, V);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            a[6 * i + j] = W[3 * i + j];
            a[6 * (3 + i) + 3 + j] = W[3 * i + j];
            a[6 * (3 + i) + j] = V[3 * i + j];
        }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double aa = 0.0;
            for (int k = 0; k < 6; ++k) aa += a[6 * i + k] * a[6 * k + j];
            J[6 * i + j] = (i == j ? 1.0 : 0.0) + 0.5 * a[6 * i + j] + aa / 12.0;
        }
}

// Shifted Tukey weight of the whitened error norm x: tukey(|x - offset|, w)
// with tukey(y, w) = (max(0, 1 - y^2 / w))^2.
double tukey_weight(double x, double w, double offset)
{
    const double y = x - offset, u = 1.0 - y * y / w;
    return u > 0.0 ? u * u : 0.0;
}

// Robust loss whose derivative in s = x^2 is that weight: rho = int_0^x weight(u) 2u du,
// by three-point Gauss-Legendre on the weight's support (exact: a degree-5 polynomial).
double tukey_loss(double x, double w, double offset)
{
    const double h = std::sqrt(w), lo = std::max(0.0, offset - h), hi = std::min(x, offset + h);
    if (!(hi > lo)) return 0.0;
    const double c = 0.5 * (lo + hi), r = 0.5 * (hi - lo), g = std::sqrt(0.6);
    const double nodes[3] = {c - r * g, c, c + r * g}, wts[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += wts[k] * tukey_weight(nodes[k], w, offset) * 2.0 * nodes[k];
    return r * s;
}

}  // namespace

extern "C" {

vgicp_status vgicp_se3_retract(double *poses, const double *delta, int64_t n_poses)
{
    if (n_poses < 0 || (n_poses > 0 && (!poses || !delta))) return VGICP_ERR_INVALID_ARG;
    for (int64_t p = 0; p < n_poses; ++p) {
        double E[12], *T = poses + 12 * p, N[12];
        se3_exp(delta + 6 * p, E);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 4; ++j) {
                double s = j == 3 ? T[4 * i + 3] : 0.0;
                for (int k = 0; k < 3; ++k) s += T[4 * i + k] * E[4 * k + j];
                N[4 * i + j] = s;
            }
        std::memcpy(T, N, sizeof(N));
    }
    return VGICP_OK;
}

vgicp_status vgicp_solve_step(const int32_t *pairs, const double *H, const double *b, int64_t n_f, int64_t n_poses,
                              int32_t anchor, double lambda, double *delta, double *model_decrease)
{
    if (n_f < 0 || n_poses <= 0 || !delta || (n_f > 0 && (!pairs || !H || !b)) || anchor < 0 || anchor >= n_poses ||
        !(lambda >= 0.0) || n_poses > (1 << 26))
        return VGICP_ERR_INVALID_ARG;
    for (int64_t f = 0; f < 2 * n_f; ++f)
        if (pairs[f] < 0 || pairs[f] >= n_poses) return VGICP_ERR_INVALID_ARG;
    // pose graph without the anchor; position of each free pose in the RCM order
    std::vector<std::vector<int>> adj((size_t)n_poses);
    for (int64_t f = 0; f < n_f; ++f) {
        const int a = pairs[2 * f], c = pairs[2 * f + 1];
        if (a != c && a != anchor && c != anchor) {
            adj[a].push_back(c);
            adj[c].push_back(a);
        }
    }
    for (auto &v : adj) {
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
    }
    adj[anchor].clear();
    std::vector<int> order = rcm_order(adj);
    order.erase(std::remove(order.begin(), order.end(), (int)anchor), order.end());
    const int64_t m = (int64_t)order.size(), nv = 6 * m;
    std::vector<int64_t> pos((size_t)n_poses, -1);
    for (int64_t i = 0; i < m; ++i) pos[order[i]] = i;
    // envelope: the first block column of each block row
    std::vector<int64_t> first_block((size_t)m);
    for (int64_t i = 0; i < m; ++i) {
        int64_t fb = i;
        for (int v : adj[order[i]]) fb = std::min(fb, pos[v]);
        first_block[i] = fb;
    }
    Skyline S;
    S.first.resize(nv);
    S.off.resize(nv + 1);
    int64_t tot = 0;
    for (int64_t r = 0; r < nv; ++r) {
        S.first[r] = 6 * first_block[r / 6];
        S.off[r] = tot;
        tot += r - S.first[r] + 1;
    }
    S.off[nv] = tot;
    S.a.assign((size_t)tot, 0.0);
    std::vector<double> rhs((size_t)nv, 0.0);
    for (int64_t f = 0; f < n_f; ++f) {
        const int32_t pose[2] = {pairs[2 * f], pairs[2 * f + 1]};
        const double *Hf = H + 144 * f, *bf = b + 12 * f;
        for (int bi = 0; bi < 2; ++bi) {
            const int64_t pi = pose[bi] == anchor ? -1 : pos[pose[bi]];
            if (pi < 0) continue;
            for (int r = 0; r < 6; ++r) rhs[6 * pi + r] -= bf[6 * bi + r];
            for (int bj = 0; bj < 2; ++bj) {
                const int64_t pj = pose[bj] == anchor ? -1 : pos[pose[bj]];
                if (pj < 0 || pj > pi) continue;   // lower blocks only (the other is its transpose)
                for (int r = 0; r < 6; ++r) {
                    const int64_t R = 6 * pi + r;
                    double *row = S.a.data() + S.off[R] + (6 * pj - S.first[R]);
                    const double *h = Hf + 12 * (6 * bi + r) + 6 * bj;
                    const int cmax = pj == pi ? r + 1 : 6;
                    for (int c = 0; c < cmax; ++c) row[c] += h[c];
                }
            }
        }
    }
    // Marquardt damping: lambda times the diagonal (floored for unconstrained directions)
    double mean_diag = 0.0;
    for (int64_t r = 0; r < nv; ++r) mean_diag += S.at(r, r);
    mean_diag = nv > 0 ? mean_diag / (double)nv : 1.0;
    const double floor_d = 1e-12 * std::max(mean_diag, 1e-300);
    for (int64_t r = 0; r < nv; ++r) {
        double &d = S.at(r, r);
        d += lambda * std::max(d, floor_d) + floor_d;
    }
    if (!vg::envelope_cholesky6(S.a.data(), S.first.data(), S.off.data(), nv)) return VGICP_ERR_NUMERIC;
    // L y = rhs, L' x = y
    std::vector<double> x(rhs);
    for (int64_t i = 0; i < nv; ++i) {
        double s = x[i];
        for (int64_t k = S.first[i]; k < i; ++k) s -= S.at(i, k) * x[k];
        x[i] = s / S.at(i, i);
    }
    for (int64_t i = nv - 1; i >= 0; --i) {
        x[i] /= S.at(i, i);
        const double xi = x[i];
        for (int64_t k = S.first[i]; k < i; ++k) x[k] -= S.at(i, k) * xi;
    }
    std::fill(delta, delta + 6 * n_poses, 0.0);
    for (int64_t i = 0; i < m; ++i)
        for (int r = 0; r < 6; ++r) delta[6 * order[i] + r] = x[6 * i + r];
    if (model_decrease) {
        // the Gauss-Newton model of the summed cost: F(d) = F + 2 b'd + d'H d
        std::vector<double> g((size_t)6 * n_poses, 0.0), Hd((size_t)6 * n_poses);
        for (int64_t f = 0; f < n_f; ++f)
            for (int bi = 0; bi < 2; ++bi)
                for (int r = 0; r < 6; ++r) g[6 * pairs[2 * f + bi] + r] += b[12 * f + 6 * bi + r];
        global_matvec(pairs, H, n_f, delta, Hd.data(), n_poses);
        double bd = 0.0, dHd = 0.0;
        for (int64_t i = 0; i < 6 * n_poses; ++i) {
            bd += g[i] * delta[i];
            dHd += delta[i] * Hd[i];
        }
        *model_decrease = -(2.0 * bd + dHd);
    }
    return VGICP_OK;
}

vgicp_status vgicp_loop_linearize(const vgicp_loop_factor *loops, int64_t n_loops, const double *poses,
                                  int64_t n_poses, double *H, double *b, double *cost)
{
    if (n_loops < 0 || (n_loops > 0 && (!loops || !poses || !cost)) || n_poses < 0) return VGICP_ERR_INVALID_ARG;
    for (int64_t l = 0; l < n_loops; ++l) {
        const vgicp_loop_factor &L = loops[l];
        if (L.pose_i < 0 || L.pose_i >= n_poses || L.pose_j < 0 || L.pose_j >= n_poses || !(L.width > 0.0))
            return VGICP_ERR_INVALID_ARG;
        // r = Log(That^-1 T_i^-1 T_j), x = sqrt(r' Omega r)
        double Ti_inv[12], D[12], Mi[12], E[12], r[6];
        invert34(poses + 12 * L.pose_i, Ti_inv);
        compose34(Ti_inv, poses + 12 * L.pose_j, D);
        invert34(L.T_ij, Mi);
        compose34(Mi, D, E);
        se3_log(E, r);
        double Or[6];
        for (int i = 0; i < 6; ++i) {
            Or[i] = 0.0;
            for (int j = 0; j < 6; ++j) Or[i] += L.information[6 * i + j] * r[j];
        }
        double s2 = 0.0;
        for (int i = 0; i < 6; ++i) s2 += r[i] * Or[i];
        const double x = std::sqrt(std::max(s2, 0.0));
        cost[l] = tukey_loss(x, L.width, L.offset);
        if (!H && !b) continue;
        const double wgt = tukey_weight(x, L.width, L.offset);
        // J_j = Jr^-1(r), J_i = -Jr^-1(r) Ad(D^-1)  (right perturbations of T_i and T_j)
        double Jinv[36], Dinv[12], Ad[36], J[6][12];
        jr_inverse(r, Jinv);
        invert34(D, Dinv);
        adjoint(Dinv, Ad);
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double s = 0.0;
                for (int k = 0; k < 6; ++k) s += Jinv[6 * i + k] * Ad[6 * k + j];
                J[i][j] = -s;
                J[i][6 + j] = Jinv[6 * i + j];
            }
        if (H)
            for (int a = 0; a < 12; ++a)
                for (int c = 0; c < 12; ++c) {
                    double s = 0.0;
                    for (int i = 0; i < 6; ++i)
                        for (int j = 0; j < 6; ++j) s += J[i][a] * L.information[6 * i + j] * J[j][c];
                    H[144 * l + 12 * a + c] = wgt * s;
                }
        if (b)
            for (int a = 0; a < 12; ++a) {
                double s = 0.0;
                for (int i = 0; i < 6; ++i) s += J[i][a] * Or[i];
                b[12 * l + a] = wgt * s;
            }
    }
    return VGICP_OK;
}

vgicp_status vgicp_optimize(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f, double *poses,
                            int64_t n_poses, const vgicp_lm_options *opt_in, vgicp_lm_report *report)
{
    return vgicp_optimize_with_loops(ctx, factors, n_f, nullptr, 0, poses, n_poses, opt_in, report);
}

vgicp_status vgicp_optimize_with_loops(vgicp_ctx *ctx, const vgicp_factor *factors, int64_t n_f,
                                       const vgicp_loop_factor *loops, int64_t n_loops, double *poses,
                                       int64_t n_poses, const vgicp_lm_options *opt_in, vgicp_lm_report *report)
{
    if (!ctx) return VGICP_ERR_INVALID_ARG;
    if (n_f <= 0 || n_poses <= 0 || !factors || !poses || n_loops < 0 || (n_loops > 0 && !loops))
        return VGICP_ERR_INVALID_ARG;
    vgicp_lm_options opt{};
    if (opt_in) opt = *opt_in;
    if (opt.max_iterations <= 0) opt.max_iterations = 20;
    if (opt.lambda_init <= 0.0) opt.lambda_init = 1e-4;
    if (opt.relative_tolerance <= 0.0) opt.relative_tolerance = 1e-6;
    if (opt.anchor < 0 || opt.anchor >= n_poses) return VGICP_ERR_INVALID_ARG;
    vgicp_lm_report rep{};
    // system rows: the matching cost factors, then the loop factors
    const int64_t n_all = n_f + n_loops;
    std::vector<int32_t> pairs((size_t)n_all * 2);
    for (int64_t f = 0; f < n_f; ++f) {
        pairs[2 * f] = factors[f].target_pose;
        pairs[2 * f + 1] = factors[f].source_pose;
    }
    for (int64_t l = 0; l < n_loops; ++l) {
        if (loops[l].pose_i < 0 || loops[l].pose_i >= n_poses || loops[l].pose_j < 0 || loops[l].pose_j >= n_poses)
            return VGICP_ERR_INVALID_ARG;
        pairs[2 * (n_f + l)] = loops[l].pose_i;
        pairs[2 * (n_f + l) + 1] = loops[l].pose_j;
    }
    vgicp_plan *plan = nullptr;
    vgicp_status st = vgicp_plan_create(ctx, factors, n_f, n_poses, &plan);
    if (st != VGICP_OK) return st;
    std::vector<double> H((size_t)n_all * 144), b((size_t)n_all * 12), cost((size_t)n_all),
        delta((size_t)n_poses * 6);
    std::vector<double> trial((size_t)n_poses * 12);
    auto sum = [](const std::vector<double> &v) {
        double s = 0.0;
        for (double x : v) s += x;
        return s;
    };
    // F and the system at `at`: matching cost factors on the GPU, loop factors on the host
    auto linearize_all = [&](const double *at) {
        vgicp_status e = vgicp_plan_linearize(ctx, plan, at, H.data(), b.data(), cost.data(), nullptr,
                                              VGICP_MEM_HOST);
        if (e == VGICP_OK && n_loops)
            e = vgicp_loop_linearize(loops, n_loops, at, n_poses, H.data() + 144 * n_f, b.data() + 12 * n_f,
                                     cost.data() + n_f);
        return e;
    };
    auto evaluate_all = [&](const double *at) {
        vgicp_status e = vgicp_evaluate(ctx, factors, n_f, at, n_poses, cost.data(), nullptr, VGICP_MEM_HOST);
        if (e == VGICP_OK && n_loops)
            e = vgicp_loop_linearize(loops, n_loops, at, n_poses, nullptr, nullptr, cost.data() + n_f);
        return e;
    };
    auto t0 = Clock::now();
    st = linearize_all(poses);
    rep.linearize_ms += ms_since(t0);
    double F = sum(cost), lambda = opt.lambda_init;
    rep.initial_cost = F;
    rep.history[rep.n_history++] = F;
    int rejects = 0;
    for (int it = 0; st == VGICP_OK && it < opt.max_iterations; ++it) {
        ++rep.iterations;
        double pred = 0.0;
        t0 = Clock::now();
        st = vgicp_solve_step(pairs.data(), H.data(), b.data(), n_all, n_poses, opt.anchor, lambda, delta.data(),
                              &pred);
        rep.solve_ms += ms_since(t0);
        if (st == VGICP_ERR_NUMERIC) {   // not positive definite at this damping: damp more
            st = VGICP_OK;
            lambda *= 10.0;
            if (++rejects > 10) break;
            continue;
        }
        if (st != VGICP_OK) break;
        if (pred <= opt.relative_tolerance * F) break;   // the model promises no further progress
        std::memcpy(trial.data(), poses, trial.size() * sizeof(double));
        vgicp_se3_retract(trial.data(), delta.data(), n_poses);
        t0 = Clock::now();
        st = evaluate_all(trial.data());
        rep.evaluate_ms += ms_since(t0);
        if (st != VGICP_OK) break;
        const double Fn = sum(cost);
        if (Fn < F) {
            ++rep.accepted;
            rejects = 0;
            std::memcpy(poses, trial.data(), trial.size() * sizeof(double));
            const double rel = (F - Fn) / std::max(F, 1e-300);
            F = Fn;
            if (rep.n_history < 64) rep.history[rep.n_history++] = F;
            lambda = std::max(lambda / 10.0, 1e-12);
            if (rel < opt.relative_tolerance) break;
            t0 = Clock::now();
            st = linearize_all(poses);
            rep.linearize_ms += ms_since(t0);
        } else {
            lambda *= 10.0;
            if (++rejects > 10) break;
        }
    }
    rep.final_cost = F;
    rep.lambda = lambda;
    vgicp_plan_destroy(ctx, plan);
    if (report) *report = rep;
    return st;
}

}  // extern "C"
