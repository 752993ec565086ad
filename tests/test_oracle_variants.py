"""Pins of the oracle's VGICP variants (no GPU): neighbour-voxel association
(DIRECT7 / DIRECT27) and count-weighted correspondences.

A hand-worked case with dyadic numbers fixes cost, inliers and the translational
parts of b exactly; a brute-force enumeration of every (point, voxel) pair in the
neighbour set, written with numpy linear algebra, checks random clouds."""
import itertools

import numpy as np
import pytest

import datagen as dg
import oracle

IDENT = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)


def _half_identity(n):
    return np.tile(np.array([0.5, 0.0, 0.0, 0.5, 0.0, 0.5], np.float32), (n, 1))


def test_hand_worked_neighbours_and_weights():
    # target voxels (r = 1): (0,0,0) holds (0.25,.5,.5); (1,0,0) holds (1.5,.5,.5) and
    # (1.75,.5,.5) (mean 1.625, count 2); (1,1,0) holds (1.5,1.5,.5).  All covariances
    # 0.5 I, so Omega = (0.5 I + 0.5 I)^-1 = I.  Source point (0.75,.5,.5), T = I.
    tgt = np.array([[0.25, 0.5, 0.5], [1.5, 0.5, 0.5], [1.75, 0.5, 0.5], [1.5, 1.5, 0.5]], np.float32)
    src = np.array([[0.75, 0.5, 0.5]], np.float32)
    vm = oracle.voxelmap(tgt, _half_identity(4), 1.0)
    e = {"own": np.array([-0.5, 0, 0]), "px": np.array([0.875, 0, 0]), "pxpy": np.array([0.75, 1.0, 0])}
    c = {k: float(v @ v) for k, v in e.items()}
    cases = [(1, False, ["own"], [1]), (7, False, ["own", "px"], [1, 1]), (7, True, ["own", "px"], [1, 2]),
             (27, False, ["own", "px", "pxpy"], [1, 1, 1]), (27, True, ["own", "px", "pxpy"], [1, 2, 1])]
    for nb, wt, names, w in cases:
        L = oracle.linearize(vm, src, _half_identity(1), IDENT, neighbors=nb, count_weighted=wt)
        assert L.inliers == len(names)
        assert L.cost == sum(wi * c[k] for k, wi in zip(names, w))
        bv = sum(wi * e[k] for k, wi in zip(names, w))
        assert np.array_equal(L.b[3:6], bv) and np.array_equal(L.b[9:12], -bv)


def _brute_force(vm, pts, covs, T, nb, weighted):
    """Every (point, voxel) pair whose voxel lies in the neighbour set of the point's
    own voxel: cost = sum w e' (C_v + R C_p R')^-1 e by numpy."""
    R, t = T[:, :3], T[:, 3]
    keys = {tuple(k): i for i, k in enumerate(vm.keys)}
    own, valid = oracle.voxel_coords(pts, vm.resolution, T)
    if nb == 1:
        offs = [(0, 0, 0)]
    elif nb == 7:
        offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    else:
        offs = list(itertools.product((-1, 0, 1), repeat=3))
    cost, n = 0.0, 0
    for i, p in enumerate(pts.astype(np.float64)):
        if not valid[i]:
            continue
        cp = covs[i].astype(np.float64)
        Cp = np.array([[cp[0], cp[1], cp[2]], [cp[1], cp[3], cp[4]], [cp[2], cp[4], cp[5]]])
        q = R @ p + t
        for o in offs:
            v = keys.get(tuple(own[i] + np.array(o)))
            if v is None:
                continue
            cv = vm.cov[v]
            Cv = np.array([[cv[0], cv[1], cv[2]], [cv[1], cv[3], cv[4]], [cv[2], cv[4], cv[5]]])
            e = vm.mu[v] - q
            w = float(vm.counts[v]) if weighted else 1.0
            cost += w * float(e @ np.linalg.solve(Cv + R @ Cp @ R.T, e))
            n += 1
    return cost, n


@pytest.mark.parametrize("nb", [1, 7, 27])
@pytest.mark.parametrize("weighted", [False, True])
def test_neighbour_costs_match_brute_force(nb, weighted):
    rng = dg.Stream(300 + nb + weighted)
    tgt = dg.sample_small_scene(rng, 400)
    src = dg.sample_small_scene(rng, 150)
    ct, cs = oracle.covariances(tgt), oracle.covariances(src)
    T = dg.random_pose(rng, 5, 0.5)
    vm = oracle.voxelmap(tgt, ct, 0.5)
    L = oracle.linearize(vm, src, cs, T, neighbors=nb, count_weighted=weighted)
    cost, n = _brute_force(vm, src, cs, T, nb, weighted)
    assert L.inliers == n
    assert L.cost == pytest.approx(cost, rel=1e-10)


def test_neighbour_sets_nest():
    rng = dg.Stream(333)
    tgt = dg.sample_small_scene(rng, 600)
    src = dg.sample_small_scene(rng, 300)
    ct, cs = oracle.covariances(tgt), oracle.covariances(src)
    T = dg.random_pose(rng, 5, 0.5)
    vm = oracle.voxelmap(tgt, ct, 1.0)
    L1, L7, L27 = (oracle.linearize(vm, src, cs, T, neighbors=nb) for nb in (1, 7, 27))
    assert L1.inliers < L7.inliers < L27.inliers
    assert L1.cost < L7.cost < L27.cost
    # count weights scale every term by a count >= 1
    W1 = oracle.linearize(vm, src, cs, T, count_weighted=True)
    assert W1.inliers == L1.inliers and W1.cost >= L1.cost
