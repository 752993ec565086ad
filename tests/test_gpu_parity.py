"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bit-exact: voxel keys and counts, per-point correspondences, overlap counts,
inlier counts, kNN neighbour-dependent identity cases.  Floating point: voxel
means within 1e-6 r and covariances within 1e-6 of their scale; cost, H and b
within err(X) = max_i |X_i - X_i^ref| / S_i <= 1e-5 (float64 path) and
<= 1e-4 (float32 path), S_i the sum of absolute per-point contributions.
"""
import numpy as np
import pytest

import datagen as dg
import oracle
import paper_2109_07073_b300 as vg
from util import err_metric

pytestmark = pytest.mark.gpu

TOL = {vg.VGICP_PREC_F32: 1e-4, vg.VGICP_PREC_F64: 1e-5, vg.VGICP_PREC_F32_COMP: 1e-4}


@pytest.fixture(scope="module")
def ctx():
    vg.load()
    c = vg.Context()
    yield c
    c.close()


@pytest.fixture(scope="module")
def single():
    w = dg.single_factor_workload()
    cb = oracle.covariances(w.points_target)
    ca = oracle.covariances(w.points_source)
    return w, cb, ca


def check_voxelmap(ctx, h, pts, covs, r):
    ref = oracle.voxelmap(pts, covs, r)
    keys, counts, mu, cov = ctx.export_voxelmap(h)
    assert keys.shape == ref.keys.shape
    assert np.array_equal(keys, ref.keys)
    assert np.array_equal(counts, ref.counts)
    assert np.max(np.abs(mu - ref.mu)) <= 1e-6 * r
    scale = max(1e-30, float(np.abs(ref.cov).max()))
    assert np.max(np.abs(cov - ref.cov)) <= 1e-6 * scale
    assert ctx.voxelmap_size(h) == ref.n_voxels


@pytest.mark.parametrize("r", [1.0, 0.25, 2.0, 0.3])
def test_voxelmap_build(ctx, single, r):
    w, cb, _ = single
    h = ctx.build_voxelmap(w.points_target, cb, r)
    check_voxelmap(ctx, h, w.points_target, cb, r)
    ctx.release(h)


def test_voxelmap_faces_negative_and_out_of_range(ctx):
    rng = dg.Stream(21)
    r = 0.5
    face = (np.round(rng.uniform(1500, -40, 40)) * r).reshape(-1, 3)
    free = rng.uniform(1500, -30, 30).reshape(-1, 3)
    far = np.array([[2 ** 20 * r, 0, 0], [-(2 ** 20) * r - 1, 0, 0], [np.nan, 1, 1]])
    pts = np.concatenate([face, free, far]).astype(np.float32)
    cov = rng.uniform(pts.shape[0] * 6, -1, 1).astype(np.float32).reshape(-1, 6)
    h = ctx.build_voxelmap(pts, cov, r)
    check_voxelmap(ctx, h, pts, cov, r)
    ctx.release(h)


def _run_pattern_clouds(r):
    """Storage orders that shape the build's runs of equal voxels within a warp:
    one voxel for every point (one claim, every other warp adds later), two
    voxels alternating (runs of one point), blocks of 33 points per voxel (runs
    across warp boundaries), and a real cloud in random order."""
    rng = dg.Stream(23)
    one = (0.25 + 0.5 * rng.uniform(3 * 5000, 0, 1)).reshape(-1, 3) * r
    two = np.concatenate([one[:2000], one[:2000] + np.array([r, 0, 0])], 1).reshape(-1, 3)
    cells = np.repeat(np.round(rng.uniform(3 * 150, -20, 20)).reshape(-1, 3), 33, axis=0)
    blocks = (cells + 0.1 + 0.8 * rng.uniform(cells.size, 0, 1).reshape(-1, 3)) * r
    w = dg.single_factor_workload()
    perm = np.argsort(rng.uniform(w.points_target.shape[0], 0, 1))
    shuffled = w.points_target[perm]
    return [c.astype(np.float32) for c in (one, two, blocks, shuffled)]


@pytest.mark.parametrize("r", [1.0, 0.3])
def test_voxelmap_build_run_patterns(r):
    """Every run pattern builds the oracle's voxelmap (keys and counts exact), in
    the given storage order and in the spatial order, with identical exports."""
    rng = dg.Stream(24)
    with vg.Context(frame_order=0) as given, vg.Context(frame_order=2) as spatial:
        for pts in _run_pattern_clouds(r):
            cov = rng.uniform(pts.shape[0] * 6, -1, 1).astype(np.float32).reshape(-1, 6)
            hg, hs = given.build_voxelmap(pts, cov, r), spatial.build_voxelmap(pts, cov, r)
            check_voxelmap(given, hg, pts, cov, r)
            for x, y in zip(given.export_voxelmap(hg), spatial.export_voxelmap(hs)):
                assert np.array_equal(x, y)
            given.release(hg)
            spatial.release(hs)


def test_batched_build_equals_single_builds(ctx, single):
    w, cb, ca = single
    fr = [ctx.add_frame(w.points_target, cb), ctx.add_frame(w.points_source, ca),
          ctx.add_frame(w.points_target[:333], cb[:333])]
    maps = ctx.build_voxelmaps(fr, 1.0)
    check_voxelmap(ctx, int(maps[0]), w.points_target, cb, 1.0)
    check_voxelmap(ctx, int(maps[1]), w.points_source, ca, 1.0)
    check_voxelmap(ctx, int(maps[2]), w.points_target[:333], cb[:333], 1.0)
    # rebuild in place at another resolution
    maps2 = ctx.build_voxelmaps(fr, 0.5, maps)
    assert np.array_equal(maps2, maps)
    check_voxelmap(ctx, int(maps[1]), w.points_source, ca, 0.5)
    for h in list(maps) + fr:
        ctx.release(int(h))


def _face_cloud(seed, n, r):
    """Points exactly on voxel faces and corners in the target frame (after T = identity rotation)."""
    rng = dg.Stream(seed)
    return (np.round(rng.uniform(3 * n, -20, 20)) * r * 0.5).reshape(-1, 3).astype(np.float32)


@pytest.mark.parametrize("r", [1.0, 0.5, 0.3])
def test_correspondences_bit_exact(ctx, single, r):
    w, cb, ca = single
    hm = ctx.build_voxelmap(w.points_target, cb, r)
    vm = oracle.voxelmap(w.points_target, cb, r)
    rng = dg.Stream(31)
    clouds = [w.points_source, _face_cloud(5, 3000, r)]
    poses = [oracle.relative_pose(w.T_target, w.T_source), dg.identity_pose(),
             dg.random_pose(rng, 60, 3.0)]
    T = dg.identity_pose()
    T[:, 3] = [r * 3, -r * 2, r]          # integer voxel shift: faces stay on faces
    poses.append(T)
    T = dg.identity_pose()
    T[:, 3] = [r * 1000, -r * 2000, r * 777]   # large shift: split translation, faces on faces
    poses.append(T)
    T = dg.random_pose(rng, 180, 1.0)
    T[:, 3] += [512.0, -300.25, 40.5]           # large translation with rotation
    poses.append(T)
    for pts in clouds:
        hf = ctx.add_frame(pts, np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (pts.shape[0], 1)))
        for P in poses:
            keys, hit = ctx.debug_correspondences(hf, hm, P)
            corr, rkeys = oracle.correspondences(vm, pts, P)
            assert np.array_equal(keys, rkeys)
            assert np.array_equal(hit, corr >= 0)
            frac, count = ctx.overlap(hf, hm, P)
            assert count == int((corr >= 0).sum()) == oracle.overlap_count(vm, pts, P)
            assert frac == count / pts.shape[0]
        ctx.release(hf)
    ctx.release(hm)


@pytest.mark.parametrize("r", [1.0, 0.5, 0.3])
def test_overlap_matrix_faces_bit_exact(ctx, single, r):
    """The overlap matrix's float32 floor (decided on the fraction of x / r) on points
    exactly on voxel faces and corners, under poses that keep them there (identity,
    whole-voxel shifts, a 1,000-voxel shift) and under rotations: every undecided
    point takes the exact path, so the counts equal the oracle's."""
    w, cb, _ = single
    vm = oracle.voxelmap(w.points_target, cb, r)
    rng = dg.Stream(33)
    srcs = [w.points_source, _face_cloud(6, 3000, r), _face_cloud(7, 2000, r)]
    poses = [dg.identity_pose()]
    T = dg.identity_pose()
    T[:, 3] = [r * 3, -r * 2, r]
    poses.append(T)
    T = dg.identity_pose()
    T[:, 3] = [r * 1000, -r * 2000, r * 777]
    poses.append(T)
    poses.append(dg.random_pose(rng, 60, 3.0))
    cov1 = lambda n: np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (n, 1))
    fr = [ctx.add_frame(p, cov1(p.shape[0])) for p in srcs]
    hm = ctx.build_voxelmap(w.points_target, cb, r)
    # every (source, pose) combination as one row of the matrix; the target at identity
    rows = [(k, T) for k in range(len(srcs)) for T in poses]
    frs = np.array([fr[k] for k, _ in rows], np.int64)
    Ps = np.stack([T for _, T in rows])
    counts = ctx.overlap_matrix(frs, np.array([hm], np.int64), Ps, dg.identity_pose()[None])
    for q, (k, T) in enumerate(rows):
        assert counts[q, 0] == oracle.overlap_count(vm, srcs[k], T), (k, q)
    for h in fr + [hm]:
        ctx.release(int(h))


def test_overlap_empty_source_is_an_error(ctx, single):
    w, cb, _ = single
    hm = ctx.build_voxelmap(w.points_target, cb, 1.0)
    he = ctx.add_frame(np.zeros((0, 3), np.float32), np.zeros((0, 6), np.float32))
    with pytest.raises(vg.VgicpError) as e:
        ctx.overlap(he, hm, dg.identity_pose())
    assert e.value.status == 4
    ctx.release(he)
    ctx.release(hm)


@pytest.fixture(scope="module")
def loop_frames():
    """Eight frames of the urban loop (64 x 1024 LiDAR, 20,000 points each): five neighbours
    and three far away, so some pairs overlap and some are provably disjoint."""
    ids = [10, 11, 12, 13, 14, 200, 201, 330]
    g = dg.graph_workload(frame_ids=ids)
    pts = [g.points[i] for i in ids]
    covs = [oracle.covariances(p) for p in pts]
    return g, ids, pts, covs


@pytest.mark.parametrize("cull", [1, 0])
def test_overlap_matrix_bit_exact(ctx, loop_frames, cull):
    g, ids, pts, covs = loop_frames
    ctx.set_options(overlap_cull=cull)
    fr = [ctx.add_frame(p, c) for p, c in zip(pts, covs)]
    maps = ctx.build_voxelmaps(fr, g.resolution)
    P = g.poses[ids]
    counts = ctx.overlap_matrix(fr, maps, P, P)
    ctx.set_options(overlap_cull=1)
    vms = [oracle.voxelmap(p, c, g.resolution) for p, c in zip(pts, covs)]
    for s in range(len(ids)):
        for t in range(len(ids)):
            T = oracle.relative_pose(P[t], P[s])
            assert counts[s, t] == oracle.overlap_count(vms[t], pts[s], T), (s, t)
    # T_i^-1 T_i is identity only up to rounding: nearly every point stays in its own voxel
    assert all(counts[i, i] >= 0.99 * pts[i].shape[0] for i in range(len(ids)))
    assert counts[0, 7] == 0 and counts[7, 0] == 0      # far apart: no correspondence
    for h in list(maps) + fr:
        ctx.release(int(h))


@pytest.mark.parametrize("far", [1.0e4, 2.5e5])
def test_overlap_matrix_far_from_origin(ctx, loop_frames, far):
    """The same frames with every pose moved far from the origin (a common rigid
    shift of 10 km or 250 km plus a rotation): the float32 pair and chunk culling keep
    their margins when the absolute translations dwarf the relative ones, and the
    counts equal the oracle's at those poses, pair by pair."""
    g, ids, pts, covs = loop_frames
    fr = [ctx.add_frame(p, c) for p, c in zip(pts, covs)]
    maps = ctx.build_voxelmaps(fr, g.resolution)
    a = 0.7
    G = np.array([[np.cos(a), -np.sin(a), 0.0, far], [np.sin(a), np.cos(a), 0.0, -0.5 * far], [0.0, 0.0, 1.0, 37.0]])
    P = np.stack([dg.compose(G, T) for T in g.poses[ids]])
    counts = ctx.overlap_matrix(fr, maps, P, P)
    vms = [oracle.voxelmap(p, c, g.resolution) for p, c in zip(pts, covs)]
    for s in range(len(ids)):
        for t in range(len(ids)):
            T = oracle.relative_pose(P[t], P[s])
            assert counts[s, t] == oracle.overlap_count(vms[t], pts[s], T), (s, t)
    assert counts[0, 1] > 0 and counts[0, 7] == 0
    for h in list(maps) + fr:
        ctx.release(int(h))


def test_overlap_matrix_presence_structures(ctx):
    """Targets whose voxel boxes select each presence structure of the overlap
    matrix: a bitmap over a small box, the compact hash table for a sparse wide
    box, and the main table for a box too wide for either."""
    rng = dg.Stream(77)
    dense = dg.sample_small_scene(rng, 4000)                        # ~20 m box: bitmap
    wide = np.concatenate([dg.sample_small_scene(rng, 600) + np.float32([dx, dy, 0])
                           for dx, dy in ((0, 0), (900, 0), (0, 900), (900, 900))]).astype(np.float32)   # compact
    huge = np.concatenate([dg.sample_small_scene(rng, 600) + np.float32([dx, 0, 0])
                           for dx in (0, 3000)]).astype(np.float32)                                   # main table
    clouds = [dense, wide, huge]
    covs = [oracle.covariances(c) for c in clouds]
    fr = [ctx.add_frame(c, v) for c, v in zip(clouds, covs)]
    maps = ctx.build_voxelmaps(fr, 1.0)
    P = np.stack([dg.identity_pose()] + [dg.random_pose(rng, 3, 0.4) for _ in range(2)])
    counts = ctx.overlap_matrix(fr, maps, P, P)
    vms = [oracle.voxelmap(c, v, 1.0) for c, v in zip(clouds, covs)]
    for si in range(3):
        for ti in range(3):
            T = oracle.relative_pose(P[ti], P[si])
            assert counts[si, ti] == oracle.overlap_count(vms[ti], clouds[si], T), (si, ti)
    assert counts[0, 1] > 0 and counts[0, 2] > 0
    for h in list(maps) + fr:
        ctx.release(int(h))


def test_add_frames_equals_single_registrations(ctx, loop_frames):
    """Frames registered in one batched call (host and device inputs, an empty frame
    among them) give the same voxelmaps, overlaps and linearisations bit for bit."""
    import torch
    g, ids, pts, covs = loop_frames
    sizes = [p.shape[0] for p in pts[:4]] + [0] + [p.shape[0] for p in pts[4:]]
    cat_p = np.concatenate(pts[:4] + [np.zeros((0, 3), np.float32)] + pts[4:])
    cat_c = np.concatenate(covs[:4] + [np.zeros((0, 6), np.float32)] + covs[4:])
    single = [ctx.add_frame(p, c) for p, c in zip(pts, covs)]
    host = list(ctx.add_frames(cat_p, cat_c, sizes))
    dev = list(ctx.add_frames(torch.from_numpy(cat_p).cuda(), torch.from_numpy(cat_c).cuda(), sizes))
    assert ctx.frame_size(host[4]) == 0 and ctx.frame_size(dev[2]) == pts[2].shape[0]
    P = g.poses[ids]
    tg, sc = [0, 1, 2, 3, 5, 6], [1, 0, 3, 2, 6, 7]
    ref = None
    for fr in (single, host[:4] + host[5:], dev[:4] + dev[5:]):
        maps = ctx.build_voxelmaps(fr, g.resolution)
        exp = [ctx.export_voxelmap(int(h)) for h in maps]
        cnt = ctx.overlap_matrix(fr, maps, P, P)
        lin = ctx.linearize(vg.make_factors(maps[tg], np.array(fr)[sc], tg, sc), P)
        if ref is None:
            ref = (exp, cnt, lin)
        else:
            for a, b in zip(exp, ref[0]):
                assert all(np.array_equal(x, y) for x, y in zip(a, b))
            assert np.array_equal(cnt, ref[1])
            assert all(np.array_equal(x, y) for x, y in zip(lin, ref[2]))
        for h in maps:
            ctx.release(int(h))
    with pytest.raises(vg.VgicpError):
        ctx.release_many([single[0], 12345678901])         # unknown handle: nothing released
    ctx.release_many(single + host + dev)


def _ragged_case(seed=41):
    """Several targets, sources of 0, 1, 31, 2047, 2048, 2049, 5000 and 12345 points."""
    rng = dg.Stream(seed)
    tg = [dg.sample_small_scene(rng, 3000) for _ in range(3)]
    sizes = [0, 1, 31, 2047, 2048, 2049, 5000, 12345]
    src = [dg.sample_small_scene(rng, n) for n in sizes]
    tcov = [oracle.covariances(p) for p in tg]
    scov = [oracle.covariances(p) if p.shape[0] else np.zeros((0, 6), np.float32) for p in src]
    poses = np.stack([dg.identity_pose()] + [dg.random_pose(rng, 5, 0.5) for _ in range(len(src) + 2)])
    factors = []
    for i in range(len(src)):
        factors.append((i % 3, i, (i + 1) % 3, 3 + i))
    return tg, tcov, src, scov, poses, factors


def _oracle_factor(vm, pts, covs, TB, TA):
    return oracle.linearize(vm, pts, covs, oracle.relative_pose(TB, TA))


@pytest.mark.parametrize("prec", [vg.VGICP_PREC_F32, vg.VGICP_PREC_F64, vg.VGICP_PREC_F32_COMP])
def test_non_finite_source_points_are_skipped_and_counted(ctx, single, prec):
    """Source points with a NaN or infinite coordinate find no voxel on either side:
    the linearisation equals the oracle's, and the overlap counts them in N (Eq. 8)
    but never as hits, for a pair and inside a matrix."""
    w, cb, ca = single
    src = w.points_source.copy()
    n = src.shape[0]
    idx = dg.Stream(41).permutation(n)[:60]
    src[idx[:20], 0] = np.nan
    src[idx[20:40], 1] = np.inf
    src[idx[40:], 2] = -np.inf
    ctx.set_options(precision=prec)
    hm = ctx.build_voxelmap(w.points_target, cb, w.resolution)
    hf = ctx.add_frame(src, ca)
    poses = np.stack([w.T_target, w.T_source])
    H, b, cost, inl = ctx.linearize(vg.make_factors([hm], [hf], [0], [1]), poses)
    vm = oracle.voxelmap(w.points_target, cb, w.resolution)
    L = _oracle_factor(vm, src, ca, w.T_target, w.T_source)
    L_finite = _oracle_factor(vm, np.delete(src, idx, axis=0), np.delete(ca, idx, axis=0), w.T_target,
                              w.T_source)
    assert inl[0] == L.inliers == L_finite.inliers > 0
    assert np.all(np.isfinite(H[0])) and np.all(np.isfinite(b[0])) and np.isfinite(cost[0])
    assert err_metric(H[0], L.H, L.SH) <= TOL[prec]
    assert err_metric(b[0], L.b, L.Sb) <= TOL[prec]
    assert abs(cost[0] - L.cost) <= TOL[prec] * L.Scost
    T = oracle.relative_pose(w.T_target, w.T_source)
    ref = oracle.overlap_count(vm, src, T)
    fr, cnt = ctx.overlap(hf, hm, T)
    assert cnt == ref and fr == ref / n
    counts = ctx.overlap_matrix([hf], [hm], poses[1:], poses[:1])
    assert counts[0, 0] == ref
    ctx.set_options(precision=vg.VGICP_PREC_F32)
    ctx.release(hm)
    ctx.release(hf)


@pytest.mark.parametrize("prec", [vg.VGICP_PREC_F32, vg.VGICP_PREC_F64, vg.VGICP_PREC_F32_COMP])
def test_linearize_single_factor(ctx, single, prec):
    w, cb, ca = single
    ctx.set_options(precision=prec)
    hm = ctx.build_voxelmap(w.points_target, cb, w.resolution)
    hf = ctx.add_frame(w.points_source, ca)
    poses = np.stack([w.T_target, w.T_source])
    f = vg.make_factors([hm], [hf], [0], [1])
    H, b, cost, inl = ctx.linearize(f, poses)
    vm = oracle.voxelmap(w.points_target, cb, w.resolution)
    L = _oracle_factor(vm, w.points_source, ca, w.T_target, w.T_source)
    assert inl[0] == L.inliers
    assert err_metric(H[0], L.H, L.SH) <= TOL[prec]
    assert err_metric(b[0], L.b, L.Sb) <= TOL[prec]
    assert abs(cost[0] - L.cost) <= TOL[prec] * L.Scost
    assert np.array_equal(H[0], H[0].T)
    ctx.set_options(precision=vg.VGICP_PREC_F32)
    ctx.release(hm)
    ctx.release(hf)


@pytest.mark.parametrize("prec", [vg.VGICP_PREC_F32, vg.VGICP_PREC_F64, vg.VGICP_PREC_F32_COMP])
@pytest.mark.parametrize("chunk", [64, 2048])
def test_linearize_ragged_batch(ctx, prec, chunk):
    tg, tcov, src, scov, poses, factors = _ragged_case()
    ctx.set_options(precision=prec, chunk_points=chunk)
    hm = [ctx.build_voxelmap(p, c, 1.0) for p, c in zip(tg, tcov)]
    hf = [ctx.add_frame(p, c) for p, c in zip(src, scov)]
    f = vg.make_factors([hm[t] for t, _, _, _ in factors], [hf[s] for _, s, _, _ in factors],
                        [a for _, _, a, _ in factors], [b for _, _, _, b in factors])
    H, b, cost, inl = ctx.linearize(f, poses)
    vms = [oracle.voxelmap(p, c, 1.0) for p, c in zip(tg, tcov)]
    for i, (t, s, pt, ps) in enumerate(factors):
        L = _oracle_factor(vms[t], src[s], scov[s], poses[pt], poses[ps])
        assert inl[i] == L.inliers, i
        if L.inliers == 0:
            assert not H[i].any() and not b[i].any() and cost[i] == 0.0
            continue
        assert err_metric(H[i], L.H, L.SH) <= TOL[prec], i
        assert err_metric(b[i], L.b, L.Sb) <= TOL[prec], i
        assert abs(cost[i] - L.cost) <= TOL[prec] * L.Scost, i
    ctx.set_options(precision=vg.VGICP_PREC_F32, chunk_points=2048)
    for h in hm + hf:
        ctx.release(h)


@pytest.mark.parametrize("prec", [vg.VGICP_PREC_F32, vg.VGICP_PREC_F64, vg.VGICP_PREC_F32_COMP])
@pytest.mark.parametrize("nb,weighted", [(7, 0), (27, 0), (1, 1), (27, 1)])
def test_linearize_neighbour_and_weighted_variants(ctx, prec, nb, weighted):
    """DIRECT7 / DIRECT27 association and count weights against the oracle's variants;
    the cost-only evaluation agrees with the linearisation's cost bit for bit."""
    tg, tcov, src, scov, poses, factors = _ragged_case(seed=49)
    ctx.set_options(precision=prec, neighbors=nb, count_weighted=weighted)
    hm = [ctx.build_voxelmap(p, c, 0.5) for p, c in zip(tg, tcov)]
    hf = [ctx.add_frame(p, c) for p, c in zip(src, scov)]
    f = vg.make_factors([hm[t] for t, _, _, _ in factors], [hf[s] for _, s, _, _ in factors],
                        [a for _, _, a, _ in factors], [b for _, _, _, b in factors])
    H, b, cost, inl = ctx.linearize(f, poses)
    c2, i2 = ctx.evaluate(f, poses)
    if prec != vg.VGICP_PREC_F64:
        assert np.array_equal(c2, cost) and np.array_equal(i2, inl)
    vms = [oracle.voxelmap(p, c, 0.5) for p, c in zip(tg, tcov)]
    for i, (t, s_, pt, ps) in enumerate(factors):
        L = oracle.linearize(vms[t], src[s_], scov[s_], oracle.relative_pose(poses[pt], poses[ps]),
                             neighbors=nb, count_weighted=bool(weighted))
        assert inl[i] == L.inliers, i
        if L.inliers == 0:
            assert not H[i].any() and cost[i] == 0.0
            continue
        assert err_metric(H[i], L.H, L.SH) <= TOL[prec], i
        assert err_metric(b[i], L.b, L.Sb) <= TOL[prec], i
        assert abs(cost[i] - L.cost) <= TOL[prec] * L.Scost, i
    ctx.set_options(precision=vg.VGICP_PREC_F32, neighbors=1, count_weighted=0)
    for h in hm + hf:
        ctx.release(h)


def test_factor_alone_equals_factor_in_batch(ctx):
    tg, tcov, src, scov, poses, factors = _ragged_case(seed=43)
    hm = [ctx.build_voxelmap(p, c, 1.0) for p, c in zip(tg, tcov)]
    hf = [ctx.add_frame(p, c) for p, c in zip(src, scov)]
    f = vg.make_factors([hm[t] for t, _, _, _ in factors], [hf[s] for _, s, _, _ in factors],
                        [a for _, _, a, _ in factors], [b for _, _, _, b in factors])
    H, b, cost, inl = ctx.linearize(f, poses)
    for i in range(len(factors)):
        H1, b1, c1, i1 = ctx.linearize(f[i:i + 1], poses)
        assert np.array_equal(H1[0], H[i]) and np.array_equal(b1[0], b[i])
        assert c1[0] == cost[i] and i1[0] == inl[i]
    for h in hm + hf:
        ctx.release(h)


def test_linearize_device_outputs_match_host_outputs(ctx, single):
    import torch
    w, cb, ca = single
    hm = ctx.build_voxelmap(w.points_target, cb, w.resolution)
    hf = ctx.add_frame(torch.from_numpy(w.points_source).cuda(), torch.from_numpy(ca).cuda())
    poses = np.stack([w.T_target, w.T_source])
    f = vg.make_factors([hm, hm], [hf, hf], [0, 1], [1, 0])
    Hh, bh, ch, ih = ctx.linearize(f, poses)
    out = (torch.zeros((2, 12, 12), dtype=torch.float64, device="cuda"),
           torch.zeros((2, 12), dtype=torch.float64, device="cuda"),
           torch.zeros(2, dtype=torch.float64, device="cuda"), torch.zeros(2, dtype=torch.int64, device="cuda"))
    ctx.linearize(f, poses, out=out)
    ctx.synchronize()
    assert np.array_equal(out[0].cpu().numpy(), Hh) and np.array_equal(out[1].cpu().numpy(), bh)
    assert np.array_equal(out[2].cpu().numpy(), ch) and np.array_equal(out[3].cpu().numpy(), ih)
    ctx.release(hm)
    ctx.release(hf)


def test_invalid_arguments_fail_cleanly(ctx, single):
    w, cb, ca = single
    hm = ctx.build_voxelmap(w.points_target, cb, 1.0)
    hf = ctx.add_frame(w.points_source, ca)
    poses = np.stack([w.T_target, w.T_source])
    with pytest.raises(vg.VgicpError) as e:
        ctx.linearize(vg.make_factors([hm], [hf], [0], [2]), poses)
    assert e.value.status == 1
    with pytest.raises(vg.VgicpError) as e:
        ctx.linearize(vg.make_factors([hf], [hf], [0], [1]), poses)
    assert e.value.status == 3
    with pytest.raises(vg.VgicpError) as e:
        ctx.build_voxelmap(w.points_target, cb, -1.0)
    assert e.value.status == 1
    with pytest.raises(vg.VgicpError) as e:
        ctx.build_voxelmap(w.points_target, cb, float("nan"))
    assert e.value.status == 1
    ctx.release(hm)
    with pytest.raises(vg.VgicpError) as e:
        ctx.release(hm)
    assert e.value.status == 3
    ctx.release(hf)


def test_knn_covariances_match_oracle(ctx, single):
    w, cb, _ = single
    g = ctx.estimate_covariances(w.points_target, 10, 1e-3)
    assert np.max(np.abs(g - cb)) <= 2e-6
    tiny = w.points_target[:5]
    assert np.array_equal(ctx.estimate_covariances(tiny, 10, 1e-3), oracle.covariances(tiny))


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6])
def test_linearize_variants_agree(ctx, variant):
    tg, tcov, src, scov, poses, factors = _ragged_case(seed=45)
    hm = [ctx.build_voxelmap(p, c, 1.0) for p, c in zip(tg, tcov)]
    hf = [ctx.add_frame(p, c) for p, c in zip(src, scov)]
    f = vg.make_factors([hm[t] for t, _, _, _ in factors], [hf[s] for _, s, _, _ in factors],
                        [a for _, _, a, _ in factors], [b for _, _, _, b in factors])
    ctx.set_options(linearize_variant=0)
    H0, b0, c0, i0 = ctx.linearize(f, poses)
    ctx.set_options(linearize_variant=variant)
    H1, b1, c1, i1 = ctx.linearize(f, poses)
    ctx.set_options(linearize_variant=0)
    # same chunks, same per-lane order: the variants differ only in scheduling
    assert np.array_equal(i0, i1)
    assert np.allclose(H0, H1, rtol=1e-5, atol=1e-9 * np.abs(H0).max())
    assert np.allclose(b0, b1, rtol=1e-5, atol=1e-9 * np.abs(b0).max())
    for h in hm + hf:
        ctx.release(h)


def test_linearize_shared_memory_maps_mixed(ctx, loop_frames):
    """Variant 6 with targets that have a shared-memory image (<= 4,096 voxels), one
    too large for it (0.25 m voxels), and an empty one: equal to variant 0 and to
    the oracle."""
    g, ids, pts, covs = loop_frames
    P = g.poses[ids]
    hm_small = [ctx.build_voxelmap(pts[i], covs[i], 1.0) for i in range(3)]
    hm_big = ctx.build_voxelmap(pts[3], covs[3], 0.25)
    hm_empty = ctx.build_voxelmap(np.zeros((0, 3), np.float32), np.zeros((0, 6), np.float32), 1.0)
    fr = [ctx.add_frame(p, c) for p, c in zip(pts[:5], covs[:5])]
    tg = [hm_small[0], hm_small[0], hm_small[1], hm_big, hm_big, hm_small[2], hm_empty]
    ti = [0, 0, 1, 3, 3, 2, 0]
    sc = [1, 2, 0, 4, 2, 1, 3]
    f = vg.make_factors(tg, np.array(fr)[sc], ti, sc)
    ctx.set_options(linearize_variant=0)
    ref = ctx.linearize(f, P)
    ctx.set_options(linearize_variant=6)
    got = ctx.linearize(f, P)
    c6, i6 = ctx.evaluate(f, P)
    ctx.set_options(linearize_variant=0)
    assert np.array_equal(got[3], ref[3])
    assert np.allclose(got[0], ref[0], rtol=1e-5, atol=1e-9 * np.abs(ref[0]).max())
    assert np.array_equal(got[2], c6) or np.allclose(got[2], c6, rtol=1e-6)
    res = {0: 1.0, 1: 1.0, 2: 1.0, 3: 0.25}
    for k in range(len(tg) - 1):
        vm = oracle.voxelmap(pts[ti[k]], covs[ti[k]], res[ti[k]])
        L = oracle.linearize(vm, pts[sc[k]], covs[sc[k]], oracle.relative_pose(P[ti[k]], P[sc[k]]))
        assert got[3][k] == L.inliers
        if L.inliers:
            assert err_metric(got[0][k], L.H, L.SH) <= TOL[vg.VGICP_PREC_F32]
    assert got[3][-1] == 0 and not got[0][-1].any()
    for h in hm_small + [hm_big, hm_empty] + fr:
        ctx.release(h)


def test_shared_memory_images_follow_rebuilds(ctx, loop_frames):
    """Images are made on first use by variant 6 and made again after a map is rebuilt
    in place (same handle): direct calls and a captured plan both see the new voxels."""
    g, ids, pts, covs = loop_frames
    P = g.poses[ids]
    fr = [ctx.add_frame(p, c) for p, c in zip(pts[:4], covs[:4])]
    maps = ctx.build_voxelmaps(fr[:2], 1.0)
    f = vg.make_factors([maps[0], maps[1], maps[0]], [fr[2], fr[3], fr[1]], [0, 1, 0], [2, 3, 1])
    ctx.set_options(linearize_variant=6)
    plan = ctx.plan_create(f, len(P))
    first = ctx.linearize(f, P)
    first_plan = ctx.plan_linearize(plan, P)
    ctx.build_voxelmaps([fr[1], fr[0]], 1.0, maps=maps)     # contents swapped, handles kept
    again = ctx.linearize(f, P)
    again_plan = ctx.plan_linearize(plan, P)
    ctx.set_options(linearize_variant=0)
    ref = ctx.linearize(f, P)
    ctx.build_voxelmaps([fr[0], fr[1]], 1.0, maps=maps)
    ref_first = ctx.linearize(f, P)
    ctx.plan_destroy(plan)
    assert not np.array_equal(ref[3], ref_first[3])
    for got, want in ((first, ref_first), (first_plan, ref_first), (again, ref), (again_plan, ref)):
        assert np.array_equal(got[3], want[3])
        assert np.allclose(got[0], want[0], rtol=1e-5, atol=1e-9 * np.abs(want[0]).max())
        assert np.allclose(got[1], want[1], rtol=1e-5, atol=1e-9 * np.abs(want[1]).max())
    for h in list(maps) + fr:
        ctx.release(h)


def test_linearize_chunk_culling_is_exact(ctx, loop_frames):
    """Skipping source chunks whose moved box misses the target's voxels changes no sum."""
    g, ids, pts, covs = loop_frames
    fr = [ctx.add_frame(p, c) for p, c in zip(pts, covs)]
    maps = ctx.build_voxelmaps(fr, g.resolution)
    P = g.poses[ids]
    tg = [0, 0, 1, 2, 3, 4, 5, 6, 0]
    sc = [1, 4, 4, 3, 0, 2, 6, 5, 7]
    f = vg.make_factors(maps[tg], np.array(fr)[sc], tg, sc)
    out = {}
    for cull in (0, 1):
        ctx.set_options(linearize_cull=cull)
        out[cull] = ctx.linearize(f, P)
    ctx.set_options(linearize_cull=1)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    vms = {t: oracle.voxelmap(pts[t], covs[t], g.resolution) for t in set(tg)}
    for k, (t, s) in enumerate(zip(tg, sc)):
        L = oracle.linearize(vms[t], pts[s], covs[s], oracle.relative_pose(P[t], P[s]))
        assert out[1][3][k] == L.inliers
        if L.inliers:
            assert err_metric(out[1][0][k], L.H, L.SH) <= TOL[vg.VGICP_PREC_F32]
    for h in list(maps) + fr:
        ctx.release(int(h))


def test_autotune_keeps_results(ctx, single):
    w, cb, ca = single
    hm = ctx.build_voxelmap(w.points_target, cb, w.resolution)
    hf = ctx.add_frame(w.points_source, ca)
    poses = np.stack([w.T_target, w.T_source])
    f = vg.make_factors([hm, hm], [hf, hf], [0, 1], [1, 0])
    best, ms = ctx.autotune(f, poses, reps=1)
    assert ms > 0 and best.linearize_variant in range(7) and best.chunk_points in (1024, 2048, 4096, 8192)
    H, b, cost, inl = ctx.linearize(f, poses)
    vm = oracle.voxelmap(w.points_target, cb, w.resolution)
    L = _oracle_factor(vm, w.points_source, ca, w.T_target, w.T_source)
    assert inl[0] == L.inliers and err_metric(H[0], L.H, L.SH) <= TOL[vg.VGICP_PREC_F32]
    ctx.set_options(linearize_variant=0, chunk_points=2048)
    ctx.release(hm)
    ctx.release(hf)


def test_knn_covariances_full_frame(ctx, loop_frames):
    """Grid kNN on a 20,000-point LiDAR frame: the same covariances as the oracle."""
    g, ids, pts, covs = loop_frames
    for p, c in zip(pts[:2], covs[:2]):
        assert np.max(np.abs(ctx.estimate_covariances(p, 10, 1e-3) - c)) <= 2e-6
    far = np.concatenate([pts[0][:3000], np.array([[900.0, 900.0, 900.0]], np.float32)])   # an isolated point
    assert np.max(np.abs(ctx.estimate_covariances(far, 10, 1e-3) - oracle.covariances(far))) <= 2e-6


def test_kernel_launch_counter_moves(ctx, single):
    w, cb, _ = single
    before = ctx.kernel_launches()
    h = ctx.build_voxelmap(w.points_target, cb, 1.0)
    assert ctx.kernel_launches() > before
    ctx.release(h)


def test_kernel_timing_records_the_hot_launches(ctx, single):
    """Each build, overlap-matrix and linearisation call adds one timed launch of
    its kernel (device milliseconds from events around the launch); a reset forgets
    them; plan runs (CUDA graphs) are not timed."""
    w, cb, ca = single
    ctx.kernel_timing_reset()
    for k in (vg.VGICP_KERNEL_LINEARIZE, vg.VGICP_KERNEL_OVERLAP_MATRIX, vg.VGICP_KERNEL_VOXELMAP_BUILD):
        assert ctx.kernel_timing(k) == (0.0, 0)
    fr = [ctx.add_frame(w.points_target, cb), ctx.add_frame(w.points_source, ca)]
    maps = ctx.build_voxelmaps(fr, 1.0)
    P = np.stack([w.T_target, w.T_source])
    for _ in range(3):
        ctx.overlap_matrix(fr, maps, P, P)
    f = vg.make_factors([maps[0]], [fr[1]], [0], [1])
    ctx.linearize(f, P)
    ctx.linearize(f, P)
    plan = ctx.plan_create(f, 2)
    ctx.plan_linearize(plan, P)
    ctx.plan_destroy(plan)
    got = {k: ctx.kernel_timing(k) for k in (vg.VGICP_KERNEL_VOXELMAP_BUILD, vg.VGICP_KERNEL_OVERLAP_MATRIX,
                                              vg.VGICP_KERNEL_LINEARIZE)}
    assert got[vg.VGICP_KERNEL_VOXELMAP_BUILD][1] == 1
    assert got[vg.VGICP_KERNEL_OVERLAP_MATRIX][1] == 3
    assert got[vg.VGICP_KERNEL_LINEARIZE][1] == 2
    assert all(ms > 0.0 for ms, _ in got.values())
    with pytest.raises(vg.VgicpError):
        ctx.kernel_timing(7)
    ctx.kernel_timing_reset()
    assert ctx.kernel_timing(vg.VGICP_KERNEL_LINEARIZE) == (0.0, 0)
    for h in list(maps) + fr:
        ctx.release(int(h))
