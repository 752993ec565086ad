"""Spatial storage order of frames (options.frame_order 1: whole frames; 2: each
4,096-point tile on its own).

Frames are stored with their points sorted by the Morton code of their cell in
a 256^3 grid over the frame's box.  Against frames stored in the given order
(frame_order = 0): voxelmaps, overlap counts and inliers are identical, H / b /
cost agree within the float32 tolerance and both meet the oracle's; the order
is deterministic (the same cloud registered in another context, alone or in a
batch of frames, gives bit-identical results); per-point outputs come back in
the given order; clouds with non-finite points, a single repeated point, or
one or two points work.
"""
import numpy as np
import pytest

import datagen as dg
import oracle
import paper_2109_07073_b300 as vg
from util import err_metric

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clouds():
    w = dg.single_factor_workload()
    cb, ca = oracle.covariances(w.points_target), oracle.covariances(w.points_source)
    rng = dg.Stream(77)
    extra = rng.uniform(3 * 500, -12, 12).reshape(-1, 3).astype(np.float32)
    src = np.concatenate([w.points_source, extra, np.array([[np.nan, 0, 0], [np.inf, 1, 1]], np.float32)])
    csrc = np.concatenate([ca, np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (extra.shape[0] + 2, 1))])
    return w, cb, src, csrc


def _run(order, w, cb, src, csrc, batch=False):
    with vg.Context(frame_order=order) as ctx:
        if batch:
            fr = ctx.add_frames(np.concatenate([w.points_target, src]), np.concatenate([cb, csrc]),
                                np.array([w.points_target.shape[0], src.shape[0]]))
            ht, hs = int(fr[0]), int(fr[1])
        else:
            ht, hs = ctx.add_frame(w.points_target, cb), ctx.add_frame(src, csrc)
        hm = ctx.build_voxelmaps([ht], 1.0)[0]
        T = oracle.relative_pose(w.T_target, w.T_source)
        f = vg.make_factors([hm], [hs], [0], [1])
        lin = ctx.linearize(f, np.stack([w.T_target, w.T_source]))
        rec = ctx.linearize_correspondences(f, np.stack([w.T_target, w.T_source]))
        ov = ctx.overlap(hs, hm, T)
        dbg = ctx.debug_correspondences(hs, hm, T)
        vox = ctx.export_voxelmap(hm)
        mat = ctx.overlap_matrix([hs, ht], [hm], np.stack([w.T_source, w.T_target]), w.T_target[None])
        return lin, rec, ov, dbg, vox, mat


@pytest.mark.parametrize("order", [1, 2])
def test_spatial_order_matches_given_order_and_oracle(clouds, order):
    w, cb, src, csrc = clouds
    a, b = _run(0, w, cb, src, csrc), _run(order, w, cb, src, csrc)
    (Ha, ba, ca_, ia), (Hb, bb, cb_, ib) = a[0], b[0]
    assert np.array_equal(ia, ib)                                     # inliers
    assert a[2] == b[2]                                               # overlap (fraction, count)
    assert np.array_equal(a[5], b[5])                                 # overlap matrix
    for x, y in zip(a[3], b[3]):                                      # per-point keys / hits, given order
        assert np.array_equal(x, y)
    # recorded correspondences: the points visited under both orders agree (which
    # points the exact group culling skips depends on how the groups are formed)
    (ka, sa), (kb, sb) = a[1][4:], b[1][4:]
    both = (sa >= 0) & (sb >= 0)
    assert np.array_equal(ka[both], kb[both]) and np.array_equal(sa[both], sb[both])
    for x, y in zip(a[4], b[4]):                                      # voxelmaps (exact sums)
        assert np.array_equal(x, y)
    vm = oracle.voxelmap(w.points_target, cb, 1.0)
    L = oracle.linearize(vm, src, csrc, oracle.relative_pose(w.T_target, w.T_source))
    corr, keys = oracle.correspondences(vm, src, oracle.relative_pose(w.T_target, w.T_source))
    assert np.all(corr[(sa < 0) | (sb < 0)] < 0)                       # a skipped point has no voxel
    assert np.array_equal(b[3][0], keys) and np.array_equal(b[3][1], corr >= 0)
    for H, bv, c, i in ((Ha, ba, ca_, ia), (Hb, bb, cb_, ib)):
        assert i[0] == L.inliers
        assert err_metric(H[0], L.H, L.SH) <= 1e-4
        assert err_metric(bv[0], L.b, L.Sb) <= 1e-4
        assert err_metric(c, [L.cost], [L.Scost]) <= 1e-4


@pytest.mark.parametrize("order", [1, 2])
def test_spatial_order_is_deterministic(clouds, order):
    w, cb, src, csrc = clouds
    one, two = _run(order, w, cb, src, csrc), _run(order, w, cb, src, csrc)
    batched = _run(order, w, cb, src, csrc, batch=True)
    for other in (two, batched):
        for x, y in zip(one[0], other[0]):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("order", [1, 2])
def test_batch_with_one_point_and_empty_frames(clouds, order):
    """A batch registration mixing ordered frames with frames of one point and of
    none (which keep the given order): every frame's overlap and debug
    association equal those of the same clouds registered one by one in the
    given order."""
    w, cb, src, csrc = clouds
    parts = [src, src[:1], src[:0], w.points_target, src[5:6]]
    covs = [csrc, csrc[:1], csrc[:0], cb, csrc[5:6]]
    T = oracle.relative_pose(w.T_target, w.T_source)
    with vg.Context(frame_order=order) as ctx, vg.Context(frame_order=0) as ref:
        hm, rm = ctx.build_voxelmap(w.points_target, cb, 1.0), ref.build_voxelmap(w.points_target, cb, 1.0)
        fr = ctx.add_frames(np.concatenate(parts), np.concatenate(covs), np.array([p.shape[0] for p in parts]))
        for h, p, c in zip(fr, parts, covs):
            r = ref.add_frame(p, c)
            assert ctx.frame_size(int(h)) == p.shape[0]
            if p.shape[0] == 0:
                continue
            assert ctx.overlap(int(h), hm, T) == ref.overlap(r, rm, T)
            for x, y in zip(ctx.debug_correspondences(int(h), hm, T), ref.debug_correspondences(r, rm, T)):
                assert np.array_equal(x, y)


@pytest.mark.parametrize("n", [1, 2, 3, 1000, 5000])
def test_spatial_order_small_and_degenerate_frames(clouds, n):
    w, cb, _, _ = clouds
    same = np.tile(w.points_source[:1], (n, 1))                      # one point repeated
    cov = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (n, 1))
    for pts in (w.points_source[:n], same):
        res = []
        for order in (0, 1, 2):
            with vg.Context(frame_order=order) as ctx:
                hm = ctx.build_voxelmap(w.points_target, cb, 1.0)
                hs = ctx.add_frame(pts, cov)
                T = oracle.relative_pose(w.T_target, w.T_source)
                res.append((ctx.overlap(hs, hm, T), ctx.debug_correspondences(hs, hm, T),
                            ctx.linearize(vg.make_factors([hm], [hs], [0], [1]), np.stack([w.T_target, w.T_source]))))
        for other in res[1:]:
            assert res[0][0] == other[0]
            assert all(np.array_equal(x, y) for x, y in zip(res[0][1], other[1]))
            assert np.array_equal(res[0][2][3], other[2][3])


def test_memory_estimate_counts_the_permutation():
    with vg.Context(frame_order=1) as a, vg.Context(frame_order=0) as b:
        n = 20000
        assert a.memory_estimate(n, False) - b.memory_estimate(n, False) == 4 * n + (-4 * n) % 256
        pts = np.zeros((n, 3), np.float32)
        cov = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (n, 1))
        a.add_frame(pts, cov)
        b.add_frame(pts, cov)
        assert a.memory_in_use() == a.memory_estimate(n, False)
        assert b.memory_in_use() == b.memory_estimate(n, False)


def test_group_culling_skips_dead_groups_exactly(clouds):
    """One cull chunk (1,024 points) holding 512 points near the target and 512
    copies 200 m away: the chunk is live, but every group of far points is dead
    by the coarse-occupancy test and is skipped, while the results equal those
    with culling off bit for bit (linearisation, recorded correspondences of the
    visited points, overlap count)."""
    w, cb, _, _ = clouds
    near = w.points_source[:512]
    src = np.concatenate([near, near + np.array([200.0, 0.0, 0.0], np.float32)]).astype(np.float32)
    cov = np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (src.shape[0], 1))
    poses = np.stack([w.T_target, w.T_source])
    T = oracle.relative_pose(w.T_target, w.T_source)
    out = {}
    for cull in (1, 0):
        with vg.Context(linearize_cull=cull, overlap_cull=cull) as ctx:
            hm = ctx.build_voxelmap(w.points_target, cb, 1.0)
            hs = ctx.add_frame(src, cov)
            f = vg.make_factors([hm], [hs], [0], [1])
            rec = ctx.linearize_correspondences(f, poses)
            cnt = ctx.overlap_matrix([hs], [hm], w.T_source[None], w.T_target[None])
            out[cull] = (rec, cnt, ctx.overlap_matrix_work())
    (H1, b1, c1, i1, k1, s1), (H0, b0, c0, i0, k0, s0) = out[1][0], out[0][0]
    assert np.array_equal(H1, H0) and np.array_equal(b1, b0) and np.array_equal(c1, c0)
    assert np.array_equal(i1, i0) and np.array_equal(out[1][1], out[0][1])
    assert np.all(s0 >= 0)                                   # culling off: every point visited
    assert np.all(s1[512:] == -1)                             # the far groups: never visited
    seen = s1 >= 0
    assert np.array_equal(k1[seen], k0[seen]) and np.array_equal(s1[seen], s0[seen])
    vm = oracle.voxelmap(w.points_target, cb, 1.0)
    corr, _ = oracle.correspondences(vm, src, T)
    assert np.all(corr[512:] < 0) and i1[0] == int((corr >= 0).sum())
    assert out[1][2][1] <= 512 < out[0][2][1] == 1024         # lookups the overlap matrix performed
