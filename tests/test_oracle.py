"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each check uses a hand-worked
closed form (Eq. 2-6 evaluated by hand on dyadic inputs, so float32 inputs are
exact), brute force, central finite differences, an invariance, the gauge null
space, an independent library routine, or a textbook special case.
"""
import json
import os

import numpy as np
import pytest

import datagen as dg
import oracle
from util import adjoint, err_metric, hat, se3_exp, to34, to44

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def single_map(mu, cov6, r):
    """Voxelmap of one point: its voxel's mean is the point and its covariance the point's."""
    return oracle.voxelmap(np.array([mu], np.float32), np.array([cov6], np.float32), r)


def diag6(a, b, c):
    return [a, 0.0, 0.0, b, 0.0, c]


EPS = 2.0 ** -10   # dyadic stand-in for the 1e-3 regulariser: float32-exact


# --------------------------------------------------------- hand-worked cases --

def test_w1_single_point_single_voxel():
    """Eq. 2-6 with T_A = T_B = I, p = 0, one target voxel.

    Omega = (C_B + C_A)^-1 = diag(1/2, 1/2, 1/(2 eps)) = diag(0.5, 0.5, 512);
    e = mu_B - 0 = (1/8, 1/4, 1/64); cost = e^T Omega e = 1/128 + 1/32 + 1/8.
    q = 0 so J = [0, I | 0, -I]: only translational blocks are non-zero."""
    vm = single_map([0.125, 0.25, 0.015625], diag6(1, 1, EPS), 1.0)
    L = oracle.linearize(vm, np.zeros((1, 3), np.float32), np.array([diag6(1, 1, EPS)], np.float32),
                         dg.identity_pose())
    assert L.inliers == 1
    # the Cholesky-based inverse rounds (sqrt 2 appears), hence 1e-14 rather than equality
    assert abs(L.cost - (1 / 128 + 1 / 32 + 1 / 8)) < 1e-14
    Om = np.diag([0.5, 0.5, 512.0])
    H = np.zeros((12, 12))
    H[3:6, 3:6] = Om
    H[9:12, 9:12] = Om
    H[3:6, 9:12] = -Om
    H[9:12, 3:6] = -Om
    np.testing.assert_allclose(L.H, H, rtol=1e-14, atol=0)
    w = [0.0625, 0.125, 8.0]
    np.testing.assert_allclose(L.b, np.array([0, 0, 0, *w, 0, 0, 0, *(-np.array(w))]), rtol=1e-14, atol=0)


def test_w1_with_non_finite_source_points():
    """W1 with three more source points, one NaN, one +inf and one -inf coordinate: they
    find no voxel, so cost, H and b keep W1's closed form, one inlier, and the overlap
    counts them in N (Eq. 8: 1 of 4)."""
    vm = single_map([0.125, 0.25, 0.015625], diag6(1, 1, EPS), 1.0)
    src = np.array([[np.nan, 0, 0], [0, 0, 0], [0, np.inf, 0], [0, 0, -np.inf]], np.float32)
    L = oracle.linearize(vm, src, np.tile(np.array(diag6(1, 1, EPS), np.float32), (4, 1)), dg.identity_pose())
    assert L.inliers == 1
    assert abs(L.cost - (1 / 128 + 1 / 32 + 1 / 8)) < 1e-14
    w = [0.0625, 0.125, 8.0]
    np.testing.assert_allclose(L.b, np.array([0, 0, 0, *w, 0, 0, 0, *(-np.array(w))]), rtol=1e-14, atol=0)
    assert np.all(np.isfinite(L.H)) and np.count_nonzero(L.H) == 12
    assert oracle.overlap_count(vm, src, dg.identity_pose()) == 1
    assert oracle.overlap(vm, src, dg.identity_pose()) == 0.25


def test_w2_lever_arm():
    """Same with r = 2, p = (1, 1/2, 1/2), e = (1/8, 1/4, 1/64): w = Omega e = (1/16, 1/8, 8),
    b_B = [q x w ; w] = (63/16, -255/32, 3/32, 1/16, 1/8, 8) and b_A = -b_B (R = I, t = 0).
    H_BB worked by hand from [q]x^T Omega [q]x, [q]x Omega, Omega; H_AA = H_BB, H_AB = -H_BB."""
    p = [1.0, 0.5, 0.5]
    vm = single_map([1.125, 0.75, 0.515625], diag6(1, 1, EPS), 2.0)
    L = oracle.linearize(vm, np.array([p], np.float32), np.array([diag6(1, 1, EPS)], np.float32),
                         dg.identity_pose())
    assert L.inliers == 1 and abs(L.cost - 0.1640625) < 1e-14
    bB = np.array([3.9375, -7.96875, 0.09375, 0.0625, 0.125, 8.0])
    np.testing.assert_allclose(L.b, np.concatenate([bB, -bB]), rtol=1e-14, atol=0)
    HBB = np.array([
        [128.125, -256.0, -0.25, 0.0, -0.25, 256.0],
        [-256.0, 512.125, -0.125, 0.25, 0.0, -512.0],
        [-0.25, -0.125, 0.625, -0.25, 0.5, 0.0],
        [0.0, 0.25, -0.25, 0.5, 0.0, 0.0],
        [-0.25, 0.0, 0.5, 0.0, 0.5, 0.0],
        [256.0, -512.0, 0.0, 0.0, 0.0, 512.0],
    ])
    np.testing.assert_allclose(L.H[:6, :6], HBB, rtol=0, atol=1e-12)
    np.testing.assert_allclose(L.H[6:, 6:], HBB, rtol=0, atol=1e-12)
    np.testing.assert_allclose(L.H[:6, 6:], -HBB, rtol=0, atol=1e-12)
    np.testing.assert_allclose(L.H[6:, :6], -HBB, rtol=0, atol=1e-12)


def test_w3_rotated_source_covariance():
    """R = Rz(90) Rx(90) sends e_z to e_x, so R C_A R^T with C_A = diag(1, 1, eps) is
    diag(eps, 1, 1) (a transposed rotation would put eps on y).  With C_B = I:
    Omega = diag(1/(1+eps), 1/2, 1/2).  p = (1,1,1), t = (1/2, 1/4, 1/8): q = (3/2, 5/4, 9/8);
    e = (1/8, 1/4, 3/8): cost = (1/64)/(1+eps) + (1/16)/2 + (9/64)/2 = 16/1025 + 13/128.
    b_A = [-(p x R^T w) ; -R^T w] with R^T w = (w_y, w_z, w_x)."""
    R = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    assert np.array_equal(R @ [0, 0, 1], [1, 0, 0])
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = [0.5, 0.25, 0.125]
    vm = single_map([1.625, 1.5, 1.5], diag6(1, 1, 1), 4.0)
    L = oracle.linearize(vm, np.ones((1, 3), np.float32), np.array([diag6(1, 1, EPS)], np.float32), T)
    assert L.inliers == 1
    assert abs(L.cost - (16 / 1025 + 13 / 128)) < 1e-15
    w = np.array([0.125 * 1024 / 1025, 0.125, 0.1875])
    Rtw = np.array([w[1], w[2], w[0]])
    bA = np.concatenate([-np.cross([1.0, 1.0, 1.0], Rtw), -Rtw])
    bB = np.concatenate([np.cross([1.5, 1.25, 1.125], w), w])
    np.testing.assert_allclose(L.b, np.concatenate([bB, bA]), rtol=0, atol=1e-15)


def test_point_to_point_special_case():
    """C_A = C_B = (sigma^2 / 2) I gives Omega = I / sigma^2: the cost is point-to-point ICP,
    sum |mu_B - q|^2 / sigma^2 over corresponding points (Segal et al. 2009, Sec. III)."""
    w = dg.single_factor_workload(n=500)
    s2 = 0.25
    cov = np.tile(np.array(diag6(s2 / 2, s2 / 2, s2 / 2), np.float32), (500, 1))
    vm = oracle.voxelmap(w.points_target, cov, 1.0)
    TBA = oracle.relative_pose(w.T_target, w.T_source)
    L = oracle.linearize(vm, w.points_source, cov, TBA)
    corr = L.corr
    q = w.points_source.astype(np.float64) @ TBA[:, :3].T + TBA[:, 3]
    e = vm.mu[corr[corr >= 0]] - q[corr >= 0]
    assert L.inliers == int((corr >= 0).sum()) > 100
    assert abs(L.cost - np.sum(e * e) / s2) < 1e-11 * L.Scost


# ------------------------------------------------------------- association --

def test_voxel_floor_faces_and_range():
    """floor semantics: a point on a face belongs to the upper voxel; keys are 21-bit signed."""
    r = 0.5
    pts = np.array([[1.0, -0.5, 0.0], [-1e-30, 0.25, 0.49999997], [2 ** 20 * r, 0, 0],
                    [-(2 ** 20) * r, 0, 0], [np.nan, 0, 0], [np.inf, 0, 0]], np.float32)
    k, v = oracle.voxel_coords(pts, r)
    assert list(v) == [True, True, False, True, False, False]
    assert k[0].tolist() == [2, -1, 0]
    assert k[1].tolist() == [-1, 0, 0]
    assert k[3].tolist() == [-(2 ** 20), 0, 0]


def _tiny_clouds(seed, n=400):
    rng = dg.Stream(seed)
    r = 0.5
    # half the points sit exactly on voxel faces, including negative coordinates
    face = (np.round(rng.uniform(3 * n // 2, -6, 6)) * r).reshape(-1, 3)
    free = rng.uniform(3 * (n - n // 2), -3, 3).reshape(-1, 3)
    pts = np.concatenate([face, free]).astype(np.float32)
    cov = np.tile(np.array(diag6(1, 1, 1e-3), np.float32), (n, 1))
    return pts, cov, r


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_lookup_binary_search_equals_linear_search(seed):
    pts, cov, r = _tiny_clouds(seed)
    vm = oracle.voxelmap(pts, cov, r)
    rng = dg.Stream(100 + seed)
    for _ in range(3):
        T = dg.random_pose(rng, 30.0, 2.0)
        corr, keys = oracle.correspondences(vm, pts, T)
        for i in range(pts.shape[0]):
            assert corr[i] == oracle.lookup(vm, keys[i], brute_force=True)


@pytest.mark.parametrize("seed", [1, 2])
def test_voxelmap_equals_bruteforce_and_direct_means(seed):
    pts, _, r = _tiny_clouds(seed)
    rng = dg.Stream(7 + seed)
    cov = rng.uniform(pts.shape[0] * 6, -1, 1).astype(np.float32).reshape(-1, 6)
    vm = oracle.voxelmap(pts, cov, r)
    bf = oracle.voxelmap(pts, cov, r, brute_force=True)
    order = np.lexsort(bf.keys.T[::-1])
    assert np.array_equal(vm.keys, bf.keys[order])
    assert np.array_equal(vm.counts, bf.counts[order])
    np.testing.assert_allclose(vm.mu, bf.mu[order], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(vm.cov, bf.cov[order], rtol=1e-12, atol=1e-12)
    # direct definition: numpy floor of p / r, group, average
    k = np.floor(pts.astype(np.float64) / r).astype(np.int64)
    for v in range(vm.n_voxels):
        m = np.all(k == vm.keys[v], axis=1)
        assert m.sum() == vm.counts[v]
        np.testing.assert_allclose(vm.mu[v], pts[m].astype(np.float64).mean(0), rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(vm.cov[v], cov[m].astype(np.float64).mean(0), rtol=1e-12, atol=1e-14)
    assert vm.counts.sum() == pts.shape[0]


def test_overlap_self_is_one_and_matches_membership():
    w = dg.single_factor_workload()
    cov = np.tile(np.array(diag6(1, 1, 1e-3), np.float32), (w.points_target.shape[0], 1))
    vm = oracle.voxelmap(w.points_target, cov, 1.0)
    assert oracle.overlap(vm, w.points_target, dg.identity_pose()) == 1.0
    T = oracle.relative_pose(w.T_target, w.T_source)
    k, v = oracle.voxel_coords(w.points_source, 1.0, T)
    keyset = set(map(tuple, vm.keys.tolist()))
    hits = sum(1 for i in range(k.shape[0]) if v[i] and tuple(k[i].tolist()) in keyset)
    assert oracle.overlap_count(vm, w.points_source, T) == hits
    far = T.copy()
    far[:, 3] += 1000.0
    assert oracle.overlap_count(vm, w.points_source, far) == 0


# -------------------------------------------------------- derivatives / FD --

@pytest.fixture(scope="module")
def factor1():
    w = dg.single_factor_workload()
    cb = oracle.covariances(w.points_target)
    ca = oracle.covariances(w.points_source)
    vm = oracle.voxelmap(w.points_target, cb, w.resolution)
    return w, vm, ca


def _rel(TB44, TA44):
    return to34(np.linalg.inv(TB44) @ TA44)


def test_jacobians_match_central_differences(factor1):
    """J = [de/dxi_B | de/dxi_A] by central differences of e = mu_B - T_BA p with
    correspondences frozen, perturbing T_B <- T_B Exp(h d) and T_A <- T_A Exp(h d)."""
    w, vm, ca = factor1
    TB, TA = to44(w.T_target), to44(w.T_source)
    TBA = oracle.relative_pose(w.T_target, w.T_source)
    L = oracle.linearize(vm, w.points_source, ca, TBA)
    corr = L.corr
    e0, J, Om = oracle.residuals(vm, w.points_source, ca, TBA, corr)
    h = 1e-6
    Jfd = np.zeros_like(J)
    for i in range(12):
        d = np.zeros(6)
        d[i % 6] = h
        if i < 6:
            Tp, Tm = _rel(TB @ se3_exp(d), TA), _rel(TB @ se3_exp(-d), TA)
        else:
            Tp, Tm = _rel(TB, TA @ se3_exp(d)), _rel(TB, TA @ se3_exp(-d))
        ep = oracle.residuals(vm, w.points_source, ca, Tp, corr)[0]
        em = oracle.residuals(vm, w.points_source, ca, Tm, corr)[0]
        Jfd[:, :, i] = (ep - em) / (2 * h)
    m = corr >= 0
    scale = np.maximum(1.0, np.abs(J[m]).max(axis=(1, 2)))[:, None, None]
    assert np.max(np.abs(J[m] - Jfd[m]) / scale) < 1e-7
    # H and b assembled from the differenced Jacobians (Eq. 5-6)
    Hfd = np.einsum("nai,nab,nbj->ij", Jfd[m], Om[m], Jfd[m])
    bfd = np.einsum("nai,nab,nb->i", Jfd[m], Om[m], e0[m])
    assert err_metric(L.H, Hfd, L.SH) < 1e-6
    assert err_metric(L.b, bfd, L.Sb) < 1e-6


def test_gradient_of_frozen_cost_is_twice_b(factor1):
    """With Omega and correspondences frozen, d/dxi sum e^T Omega e = 2 J^T Omega e = 2 b."""
    w, vm, ca = factor1
    TB, TA = to44(w.T_target), to44(w.T_source)
    TBA = oracle.relative_pose(w.T_target, w.T_source)
    L = oracle.linearize(vm, w.points_source, ca, TBA)
    _, _, Om = oracle.residuals(vm, w.points_source, ca, TBA, L.corr)

    def f(T):
        e = oracle.residuals(vm, w.points_source, ca, T, L.corr)[0]
        return float(np.einsum("na,nab,nb->", e, Om, e))

    assert abs(f(TBA) - L.cost) <= 1e-12 * L.Scost
    h = 1e-6
    g = np.zeros(12)
    for i in range(12):
        d = np.zeros(6)
        d[i % 6] = h
        if i < 6:
            g[i] = (f(_rel(TB @ se3_exp(d), TA)) - f(_rel(TB @ se3_exp(-d), TA))) / (2 * h)
        else:
            g[i] = (f(_rel(TB, TA @ se3_exp(d))) - f(_rel(TB, TA @ se3_exp(-d)))) / (2 * h)
    assert err_metric(g, 2 * L.b, 2 * L.Sb) < 1e-6


def test_h_symmetric_psd_with_six_dim_gauge(factor1):
    """J_A = -J_B Ad(T_BA), so H [Ad xi; xi] = 0 and b . [Ad xi; xi] = 0 for all xi: rank H <= 6."""
    w, vm, ca = factor1
    TBA = oracle.relative_pose(w.T_target, w.T_source)
    L = oracle.linearize(vm, w.points_source, ca, TBA)
    assert np.array_equal(L.H, L.H.T)
    ev = np.linalg.eigvalsh(L.H)
    assert ev.min() >= -1e-12 * ev.max()
    assert int(np.sum(np.abs(ev) < 1e-9 * ev.max())) == 6
    N = np.vstack([adjoint(TBA), np.eye(6)])
    assert np.abs(L.H @ N).max() < 1e-10 * np.abs(L.H).max()
    assert np.abs(L.b @ N).max() < 1e-10 * np.abs(L.Sb).max() * 10


def test_invariance_under_common_rigid_transform(factor1):
    w, vm, ca = factor1
    TBA = oracle.relative_pose(w.T_target, w.T_source)
    L = oracle.linearize(vm, w.points_source, ca, TBA)
    # sign-flip rotation: every product in T_BA is unchanged, so results are bit-identical
    G = np.zeros((3, 4))
    G[:, :3] = np.diag([-1.0, -1.0, 1.0])
    T2 = oracle.relative_pose(dg.compose(G, w.T_target), dg.compose(G, w.T_source))
    assert np.array_equal(T2, TBA)
    L2 = oracle.linearize(vm, w.points_source, ca, T2)
    assert L2.cost == L.cost and np.array_equal(L2.H, L.H) and np.array_equal(L2.b, L.b)
    # generic rigid transform: equal to rounding
    rng = dg.Stream(99)
    for _ in range(3):
        G = dg.random_pose(rng, 180.0, 50.0)
        T3 = oracle.relative_pose(dg.compose(G, w.T_target), dg.compose(G, w.T_source))
        L3 = oracle.linearize(vm, w.points_source, ca, T3)
        assert np.array_equal(L3.corr, L.corr)
        assert abs(L3.cost - L.cost) < 1e-9 * L.Scost
        assert err_metric(L3.H, L.H, L.SH) < 1e-9 and err_metric(L3.b, L.b, L.Sb) < 1e-9


def test_relative_pose_matches_matrix_inverse():
    rng = dg.Stream(5)
    for _ in range(10):
        TB, TA = dg.random_pose(rng, 180, 500), dg.random_pose(rng, 180, 500)
        ref = np.linalg.inv(to44(TB)) @ to44(TA)
        np.testing.assert_allclose(oracle.relative_pose(TB, TA), ref[:3], rtol=0, atol=1e-12)
    T = dg.random_pose(rng, 180, 500)
    np.testing.assert_allclose(oracle.relative_pose(T, T), np.eye(4)[:3], rtol=0, atol=1e-13)


# -------------------------------------------------------- kNN covariances --

def _knn_numpy(pts, k):
    p = pts.astype(np.float64)
    out = np.zeros((p.shape[0], k), np.int64)
    for i in range(p.shape[0]):
        d = p - p[i]
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        out[i] = np.lexsort((np.arange(p.shape[0]), d2))[:k]
    return out


def test_knn_bruteforce_matches_numpy_with_ties():
    # integer lattice with duplicates: many exact distance ties, broken by lower index
    rng = dg.Stream(3)
    pts = np.floor(rng.uniform(600, 0, 5)).reshape(-1, 3).astype(np.float32)
    assert np.array_equal(oracle.knn(pts, 10, brute_force=True), _knn_numpy(pts, 10))


@pytest.mark.parametrize("cell", [0.3, 1.0, 4.0])
def test_knn_grid_matches_bruteforce(cell):
    w = dg.single_factor_workload()
    pts = np.concatenate([w.points_target, w.points_target[:50]])   # duplicates too
    assert np.array_equal(oracle.knn(pts, 10, cell=cell), oracle.knn(pts, 10, brute_force=True))
    rng = dg.Stream(4)
    lat = np.floor(rng.uniform(900, 0, 6)).reshape(-1, 3).astype(np.float32)
    assert np.array_equal(oracle.knn(lat, 10, cell=cell), oracle.knn(lat, 10, brute_force=True))
    # an isolated point far from the rest: the shell search gives up and scans
    far = np.concatenate([w.points_target[:500], np.array([[900.0, 900.0, 900.0]], np.float32)])
    assert np.array_equal(oracle.knn(far, 10, cell=cell), oracle.knn(far, 10, brute_force=True))


def test_jacobi_diagonal_and_random_spectra():
    w, V = oracle.jacobi_eig3(np.diag([3.0, -1.0, 2.0]))
    assert np.array_equal(w, [3.0, -1.0, 2.0]) and np.array_equal(V, np.eye(3))
    rng = dg.Stream(8)
    for _ in range(50):
        Q = dg.so3_exp(rng.normal(3))
        lam = rng.normal(3) * 10.0 ** rng.uniform(1, -3, 3)[0]
        A = Q @ np.diag(lam) @ Q.T
        A = 0.5 * (A + A.T)
        w, V = oracle.jacobi_eig3(A)
        s = np.abs(lam).max()
        np.testing.assert_allclose(np.sort(w), np.sort(lam), rtol=0, atol=1e-13 * s)
        np.testing.assert_allclose(np.sort(w), np.linalg.eigvalsh(A), rtol=0, atol=1e-13 * s)
        np.testing.assert_allclose(V.T @ V, np.eye(3), rtol=0, atol=1e-14)
        np.testing.assert_allclose(A @ V, V * w, rtol=0, atol=1e-13 * s)


def test_covariance_regularised_to_surface_normal():
    """Points on a plane: the normal gets eps, in-plane directions get 1."""
    rng = dg.Stream(11)
    n = dg.so3_exp([0.3, -0.5, 0.2]) @ [0, 0, 1.0]
    u = np.cross(n, [1.0, 0, 0])
    u /= np.linalg.norm(u)
    v = np.cross(n, u)
    a, b = rng.uniform(800, -3, 3), rng.uniform(800, -3, 3)
    pts = (a[:, None] * u + b[:, None] * v + 5.0).astype(np.float32)
    cov = oracle.covariances(pts, 10, 1e-3).astype(np.float64)
    for c in cov[::37]:
        C = np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])
        np.testing.assert_allclose(C @ n, 1e-3 * n, atol=2e-4)
        np.testing.assert_allclose(C @ u, u, atol=2e-4)
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(C)), [1e-3, 1, 1], atol=1e-6)


# ------------------------------------------------------------- regression --

def test_golden_single_factor_regression():
    """Oracle output on the single-factor workload, stored by tests/golden/make_golden.py
    (which calls only the oracle and the generator): guards against unjustified drift."""
    with open(os.path.join(GOLDEN, "single_factor.json")) as f:
        g = json.load(f)
    w = dg.single_factor_workload()
    cb = oracle.covariances(w.points_target)
    ca = oracle.covariances(w.points_source)
    vm = oracle.voxelmap(w.points_target, cb, w.resolution)
    TBA = oracle.relative_pose(w.T_target, w.T_source)
    L = oracle.linearize(vm, w.points_source, ca, TBA)
    assert vm.n_voxels == g["n_voxels"]
    assert L.inliers == g["inliers"]
    assert oracle.overlap_count(vm, w.points_source, TBA) == g["overlap_count"]
    np.testing.assert_allclose(L.cost, g["cost"], rtol=1e-12)
    np.testing.assert_allclose(L.b, g["b"], rtol=1e-10, atol=1e-10 * np.abs(L.Sb).max())
    np.testing.assert_allclose(np.diag(L.H), g["H_diag"], rtol=1e-10)
